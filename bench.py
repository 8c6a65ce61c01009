"""Benchmark of the encrypted 1:N match (membership, N=2^16, K=2^15, ell=512).

One step = one encrypted membership query through the whole hot path:
hoisted baby-step rotations, diagonal MAC over the pre-rotated template
diagonals, rescale, giant-step rotations, degree-59 Chebyshev threshold,
RotateAndSum. `value` is templates matched per second (K / step time) with
the query already resident in HBM; `e2e` runs the same step through the C ABI
from a host-resident query ciphertext to the exported result (one H2D and one
D2H copy per step inside the timed region).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun, one process per GPU) runs independent replicas: the
query path does not shard within one match.
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

METRIC = "templates matched/sec and p50/p99 encrypted query latency at N=2^16, K=2^15; HBM GB/s"
UNIT = "templates/s"
# the library's profiling regions (fr_profile_read) and the stages of a membership match
REGIONS = ("ntt", "modup", "ip", "moddown", "rescale", "tensor", "mac", "misc", "copy")
STAGES = ("babies", "mac", "giants", "cheb", "sum")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle: whole membership queries, timed
# ---------------------------------------------------------------------------
def oracle_queries(cfgname, T, q, seed_key, seed_enc, lq, budget_s=0.0, max_queries=1, sum_radix=8, hoist=True,
                   babies_pq=False, hoist_sum=False):
    """Time whole membership queries of the CPU oracle (the same match the library computes,
    bit for bit: on-demand BSGS at working level lq, with the bench's choices of hoisting and
    RotateAndSum radix passed in). Key generation and encryption happen before the timed region;
    the oracle derives each rotation key inside the query, as it stands. Runs one query, then
    more while the time spent stays under budget_s, at most max_queries.
    Returns (seconds per query list, threads used, membership ciphertext of the first query)."""
    import oracle
    from paper_2604_00546_gb300 import workloads as W
    c = W.CONFIGS[cfgname] if isinstance(cfgname, str) else cfgname
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(seed_key)
    oq = ok.encrypt(np.tile(q, oc.n // c["ell"]), seed_enc)
    secs, first = [], None
    while True:
        t0 = time.perf_counter()
        ref, lvl = ok.match(oq, T, c["ell"], c["n1"], 2, c["cheb_degree"], c["threshold"], level=lq,
                            sum_radix=sum_radix, hoist=hoist, babies_pq=babies_pq, hoist_sum=hoist_sum)
        secs.append(time.perf_counter() - t0)
        if first is None:
            first = (ref[0], lvl)
        if len(secs) >= max_queries or sum(secs) + secs[-1] > budget_s:
            break
    return secs, oracle.get_threads(), first


def K_over(K, latency):
    return K / latency


def max_over_ranks(x, dist=None, device=None):
    """Largest value of x over all ranks (x itself on one process)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world_size, units_per_rank, max_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world_size * units_per_rank / (max_ms / 1000.0)


# ---------------------------------------------------------------------------
def run_serving(args):
    """Serving loop: Poisson arrivals (20 req/s by default) for --serve-seconds, 70%
    membership / 30% identification, each against one of 8 resident databases
    (K in {2^12, 2^14, 2^15, 2^16, 2^17, 2^18}), N=2^16 at the working level. Requests
    are submitted at their arrival times from a producer thread through fr_match_submit
    (host-resident query ciphertexts, so every request crosses the bus) and collected
    with fr_match_poll; latency is submission to the end of the request's batch on the
    device. value = templates matched per second over the whole run."""
    import threading as th

    import torch

    from numpy.polynomial import chebyshev as npc
    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    cfg = "membership"
    c = W.CONFIGS[cfg]
    ctx = fr.Context(device=local, **W.ctx_params(cfg, level_mode=args.level_mode), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum, hoist_giants=args.hoist_giants,
                     hoist_babies=args.hoist_babies)
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(cfg))
    ctx.load_keys(keys)
    Ts = W.serving_databases(c["ell"])
    dbs = [ctx.load_db(T) for T in Ts]
    qv = W.serving_queries(16, c["ell"])
    qcts = [ctx.encrypt(keys, v, W.enc_seed(cfg, 100 + i)) for i, v in enumerate(qv)]
    reqs = W.serving_requests(args.serve_seconds, args.serve_rate)
    # warm-up: one request per (database, mode) class through the loop
    ctx.serve_start(max_batch=args.serve_batch, slots=args.serve_slots)
    warm = [ctx.submit(dbs[d], qcts[0], m) for d in range(len(dbs)) for m in (1, 2)]
    for t in warm:
        ctx.poll(t)
    torch.cuda.synchronize()
    st0 = ctx.serve_stats()
    sampler = ClockSampler(local)
    sampler.start()
    tickets = [None] * len(reqs)
    t0 = time.perf_counter() + 0.2

    def producer():
        for i, (ta, mode, d, qi) in enumerate(reqs):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = ctx.submit(dbs[d], qcts[qi], mode)

    pt = th.Thread(target=producer)
    pt.start()
    lat, checks = [], []
    t_last = t0
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0005)
        outs, ms = ctx.poll(tickets[i], -1, with_latency=True)
        t_last = time.perf_counter()
        lat.append(ms)
        ta, mode, d, qi = reqs[i]
        if mode == 2 and len(checks) < 4:
            s = Ts[d].astype(np.float64) @ qv[qi]
            n = 1 << (c["log_n"] - 1)
            sp = np.zeros(((len(s) + n - 1) // n) * n)
            sp[: len(s)] = s
            pref = npc.chebval(sp, fr.cheb_coeffs(c["cheb_degree"], c["threshold"])).sum()
            checks.append(abs(float(ctx.decrypt(keys, outs[0])[0]) - pref))
        del outs
    pt.join()
    clocks = sampler.stop()
    st1 = ctx.serve_stats()
    ctx.serve_stop()
    wall = t_last - t0
    templates = sum(len(Ts[d]) for _, _, d, _ in reqs)
    n_mem = sum(1 for r in reqs if r[1] == 2)
    batches = st1["batches"] - st0["batches"]
    line = {
        "metric": "serving loop: templates matched/s and p50/p99 request latency (Poisson arrivals, 8 databases)",
        "value": templates / wall, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "replicas",
        "dtype": "u64", "data": "synthetic (seeded Gaussian L2-normalised templates and queries)",
        "config": {"workload": "serving N=2^16 ell=512 deg59 work level %d, %d req/s for %g s, 70%% membership / "
                               "30%% identification, 8 databases K in {2^12..2^18}" % (ctx.work_level, args.serve_rate,
                                                                                         args.serve_seconds),
                   "max_batch": args.serve_batch, "slots": args.serve_slots,
                   "database_K": [len(T) for T in Ts]},
        "requests": len(reqs), "membership_requests": n_mem, "wall_s": wall,
        "requests_per_s": len(reqs) / wall,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(np.mean(lat)), "max": float(np.max(lat))},
        "batches": batches, "mean_batch": len(reqs) / max(1, batches),
        "max_concurrent_batches": st1["max_concurrent_batches"],
        "membership_abs_err_sample": checks, "clocks": clocks,
    }
    return line


def run_identify(args):
    """Identification at scale: K=2^20 templates (32 groups of 2^15), N=2^16 at the working
    level, degree-59 threshold per slot. The database is kept as FP32 templates (2 GB) and
    every query encodes the 2^14 pre-rotated diagonals of all groups on the device (tier C)
    unless --identify-tier 1 stores them. Times one query per step with CUDA events and
    checks the decisions of every slot against the FP64 scores outside the 0.02 margin."""
    import torch

    from numpy.polynomial import chebyshev as npc
    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(device=torch.device("cuda", local))
    cfg = "identify"
    c = W.CONFIGS[cfg]
    T, q, planted = W.workload(cfg)
    K = len(T)
    ctx = fr.Context(device=local, cuda_stream=stream.cuda_stream, db_tier=args.identify_tier,
                     **W.ctx_params(cfg, level_mode=args.level_mode), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum, hoist_giants=args.hoist_giants,
                     hoist_babies=args.hoist_babies)
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_IDENTIFY), W.key_seed(cfg))
    ctx.load_keys(keys)
    db = ctx.load_db(T)
    info = db.info()
    dq = ctx.encrypt(keys, q, W.enc_seed(cfg)).upload()
    for _ in range(2):
        out = ctx.match(db, dq, fr.FR_MODE_IDENTIFY)
    ctx.sync()
    s = T.astype(np.float64) @ q
    dec = np.concatenate([ctx.decrypt(keys, o) for o in out])[:K]
    p = npc.chebval(s, fr.cheb_coeffs(c["cheb_degree"], c["threshold"]))
    far = np.abs(s - 0.5) > 0.02
    agree = bool(np.array_equal((dec >= 0.5)[far], (s >= 0.5)[far]))
    found = set(np.nonzero(dec >= 0.5)[0].tolist())
    del out
    steps = max(1, args.steps // 3)
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    outs = [ctx.match(db, dq, fr.FR_MODE_IDENTIFY) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / steps
    del outs
    # one eager profiled query: device time per region and per stage
    ctx.profile(True)
    outs = ctx.match(db, dq, fr.FR_MODE_IDENTIFY)
    torch.cuda.synchronize()
    regions = {r: ctx.profile_read(r)[0] for r in ("ntt", "modup", "ip", "moddown", "rescale", "tensor", "mac",
                                                   "misc", "encode")}
    stages = {st: ctx.profile_read("stage:" + st)[0] for st in ("babies", "encode", "mac", "giants", "cheb")}
    ntt_bytes = ctx.profile_read("ntt")[2]
    ctx.profile(False)
    del outs
    # the encoder against the measured FP64 rate: 5 n log2 n operations per diagonal FFT
    # (n = N/2 complex points), G ell diagonals per query when they are encoded per query
    n = 1 << (c["log_n"] - 1)
    fft_ops = 5.0 * n * (c["log_n"] - 1) * info["groups"] * c["ell"] if info["tier"] == 2 else 0.0
    fp64 = fr.fp64_peak(local) / 1e9
    roofline = None
    if fft_ops and regions["encode"] > 0:
        ach = fft_ops / (regions["encode"] / 1000.0) / 1e9
        roofline = {"kernel": "encoder (gather, FP64 special FFT, rounding to residues)", "bound": "fp64",
                    "achieved": ach, "peak": fp64, "unit": "GFLOP/s", "frac": ach / fp64 if fp64 else None,
                    "flops_per_query": fft_ops, "peak_kind": "measured: register-only FP64 FMA loop (fr_fp64_peak)"}
    # the NTTs against the measured butterfly rate (the region counts 16 B per coefficient)
    bfly = fr.butterfly_peak(local) / 1e9
    ntt_g = (ntt_bytes / 16.0 * (c["log_n"] / 2.0)) / (regions["ntt"] / 1000.0) / 1e9 if regions["ntt"] > 0 else 0.0
    ntt_view = {"achieved": ntt_g, "peak": bfly, "unit": "Gbutterfly/s", "frac": ntt_g / bfly if bfly else None,
                "bound": "alu", "peak_kind": "measured: register-only butterfly loop (fr_butterfly_peak)"}
    line = {
        "metric": "identification: templates matched/s and query latency at N=2^16, K=2^20",
        "value": K / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": steps, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "u64",
        "data": "synthetic (seeded Gaussian L2-normalised templates, 32 planted duplicates at cosine 0.8)",
        "config": {"workload": "identify N=2^16 K=2^20 ell=512 n1=32 deg59", "K": K, "groups": info["groups"],
                   "tier": {1: "stored diagonals", 2: "per-query diagonal encoding on device",
                            3: "stored integer coefficients, per-query residues and NTT"}[info["tier"]],
                   "work_level": ctx.work_level, "db_bytes": info["bytes"]},
        "check": {"max_abs_err_threshold": float(np.abs(dec - p).max()), "decisions_agree_outside_margin": agree,
                  "planted_found": int(len(set(planted.tolist()) & found)), "planted": int(len(planted))},
        "regions_ms": regions, "stages_ms": stages,
        "roofline": roofline, "ntt_alu": ntt_view,
        "clocks": clocks,
    }
    return line


def run_multi(args):
    """Batched launches: 64 encrypted queries (ell=512), each against its own database, with
    K_d drawn log-uniformly in [2^10, 2^17] (seeded Gaussian, L2-normalised), N=2^16 at the
    working level, membership mode. The storage tier of each database is chosen by the
    library's planner under an HBM budget (stored diagonals while they fit, then stored
    coefficients, then per-query encoding). Times one fr_match_multi over the 64 pairs
    (graph replay) against the 64 matches run one by one, and checks sampled outputs against
    the FP64 membership sums."""
    import torch

    from numpy.polynomial import chebyshev as npc
    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(device=torch.device("cuda", local))
    cfg = "membership"
    c = W.CONFIGS[cfg]
    ctx = fr.Context(device=local, cuda_stream=stream.cuda_stream, **W.ctx_params(cfg, level_mode=args.level_mode), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum, hoist_giants=args.hoist_giants,
                     hoist_babies=args.hoist_babies)
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(cfg))
    ctx.load_keys(keys)
    sizes = W.multi_sizes(args.multi_n)
    Ts = [W.multi_database(d, K, c["ell"]) for d, K in enumerate(sizes)]
    # storage plan: stored diagonals for the largest databases within the budget, stored
    # integer coefficients (1/(level+1) of that) for the rest
    n = 1 << (c["log_n"] - 1)
    group_bytes = c["ell"] * (ctx.work_level + 1) * (1 << c["log_n"]) * 8
    plan, used = {}, 0.0
    for d in sorted(range(len(sizes)), key=lambda d: -sizes[d]):
        gb = ((sizes[d] + n - 1) // n) * group_bytes / 2**30
        plan[d] = 1 if used + gb <= args.multi_budget_gb else 3
        used += gb if plan[d] == 1 else 0.0
    dbs = [ctx.load_db(T, tier=plan[d]) for d, T in enumerate(Ts)]
    tiers = [d.info()["tier"] for d in dbs]
    qv = W.serving_queries(args.multi_n, c["ell"], seed=W.MULTI_SEED + 7)
    qs = [ctx.encrypt(keys, v, W.enc_seed(cfg, 200 + i)).upload() for i, v in enumerate(qv)]
    # kernels launched per call for both forms: a 64-query graph would hold its own copy of
    # the batch's workspace (tens of GB) next to the stream-ordered pool
    ctx.use_graphs(False)
    for _ in range(2):
        outs = ctx.match_multi(dbs, qs, fr.FR_MODE_MEMBERSHIP)
    ctx.sync()
    errs = []
    for b in range(0, args.multi_n, max(1, args.multi_n // 4)):
        s = Ts[b].astype(np.float64) @ qv[b]
        sp = np.zeros(((len(s) + n - 1) // n) * n)
        sp[: len(s)] = s
        pref = npc.chebval(sp, fr.cheb_coeffs(c["cheb_degree"], c["threshold"])).sum()
        errs.append(abs(float(ctx.decrypt(keys, outs[b][0])[0]) - pref))
    del outs
    steps = max(2, args.steps // 5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    e0.record(stream)
    outs = [ctx.match_multi(dbs, qs, fr.FR_MODE_MEMBERSHIP) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / steps
    del outs
    # the same 64 pairs one match at a time
    for _ in range(1):
        outs = [ctx.match(d, q, fr.FR_MODE_MEMBERSHIP) for d, q in zip(dbs, qs)]
    torch.cuda.synchronize()
    e0.record(stream)
    outs = [ctx.match(d, q, fr.FR_MODE_MEMBERSHIP) for d, q in zip(dbs, qs)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1)
    del outs
    total = sum(sizes)
    line = {
        "metric": "batched launches: templates matched/s, 64 queries against 64 databases of uneven sizes",
        "value": total / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": steps, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "u64", "data": "synthetic (seeded Gaussian L2-normalised templates)",
        "config": {"workload": "multi N=2^16 ell=512 deg59 work level %d, %d queries, K_d log-uniform in [2^10, 2^17]"
                               % (ctx.work_level, args.multi_n),
                   "templates": total, "groups": sum(d.info()["groups"] for d in dbs),
                   "tiers": {str(t): tiers.count(t) for t in sorted(set(tiers))},
                   "hbm_budget_gb": args.multi_budget_gb},
        "form": "kernels launched per call (programmatic dependent launch), no CUDA graph",
        "one_by_one": {"ms": ms_single, "value": total / (ms_single / 1000.0), "unit": UNIT},
        "membership_abs_err_sample": errs, "clocks": clocks,
    }
    return line


def run_encrypted(args):
    """Encrypted database (the paper's setting; enroller-side pre-rotation, lazy
    relinearisation): membership of one encrypted query against K = 2^15 encrypted templates
    (ell = 512, 32 near-duplicates), N = 2^16 at the working level. The enroller's 512
    diagonal ciphertexts are made on the host (fr_encrypt_db) and loaded as storage tier 4.
    Times one query (graph replay) and a batch of --batch queries against the same database
    held as plaintext diagonals (tier 1), reports the ct x ct MAC's HBM rate from the library's
    per-launch events, and checks the membership sum against FP64."""
    import torch

    from numpy.polynomial import chebyshev as npc
    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(device=torch.device("cuda", local))
    cfg = dict(W.CONFIGS["membership"], ell=args.db_ell)   # --db-ell: a smaller case for profiling
    c = cfg
    ctx = fr.Context(device=local, cuda_stream=stream.cuda_stream, **W.ctx_params(cfg, level_mode=args.level_mode), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum, hoist_giants=args.hoist_giants)
    # with the negative giant-step keys of the server-side pre-rotation variant
    rots = set(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP))
    rots |= set(fr.rotation_set(c["ell"], c["n1"], ctx.n, fr.FR_KEYS_TBS_TOTAL, True))
    keys = ctx.keygen(sorted(rots), W.key_seed(cfg))
    ctx.load_keys(keys)
    T, q, planted = W.workload(cfg)
    K = len(T)
    t0 = time.perf_counter()
    E = ctx.encrypt_db(keys, T, seed=0xE2000)
    enroll_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    db = ctx.load_db_encrypted(E, K)
    load_s = time.perf_counter() - t0
    del E
    dbp = ctx.load_db(T, tier=1)
    qct = ctx.encrypt(keys, q, W.enc_seed(cfg)).upload()
    mode = fr.FR_MODE_MEMBERSHIP

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            outs = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = [fn() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, outs[-1]

    sampler = ClockSampler(local)
    sampler.start()
    ms, outs = timed(lambda: ctx.match(db, qct, mode), args.steps)
    clocks = sampler.stop()
    s = T.astype(np.float64) @ q
    pref = npc.chebval(s, fr.cheb_coeffs(c["cheb_degree"], c["threshold"])).sum()
    err = abs(float(ctx.decrypt(keys, outs[0])[0]) - pref)
    del outs
    ms_pt, outs = timed(lambda: ctx.match(dbp, qct, mode), args.steps)
    del outs
    # server-side pre-rotation: plain diagonals enrolled, rotated by -j n1 at load
    Ep = ctx.encrypt_db(keys, T, seed=0xE3000, prerotate=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dbs_ = ctx.load_db_encrypted(Ep, K, prerotated=False)
    load_tbs_s = time.perf_counter() - t0
    del Ep
    ms_tbs, outs = timed(lambda: ctx.match(dbs_, qct, mode), args.steps)
    err_tbs = abs(float(ctx.decrypt(keys, outs[0])[0]) - pref)
    del outs, dbs_
    B = max(1, args.batch)
    qb = [ctx.encrypt(keys, q, W.enc_seed(cfg, 300 + i)).upload() for i in range(B)]
    ms_b, outs = timed(lambda: ctx.match_batch(db, qb, mode), max(2, args.steps // 4))
    del outs
    # per-region device time, one eager pass
    ctx.profile(True)
    outs = ctx.match(db, qct, mode)
    torch.cuda.synchronize()
    mac_ms, mac_n, mac_b = ctx.profile_read("mac")
    stages = {st: ctx.profile_read("stage:" + st)[0] for st in ("babies", "mac", "relin", "giants", "cheb", "sum")}
    ctx.profile(False)
    del outs
    hbm, hbm_src = load_peaks()
    mac_gbs = mac_b / (mac_ms / 1000.0) / 1e9 if mac_ms > 0 else None
    line = {
        "metric": "encrypted-database membership: templates matched/s (1:N, encrypted query and templates)",
        "value": K / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "u64",
        "data": "synthetic (seeded Gaussian L2-normalised templates, 32 near-duplicates at cosine 0.8)",
        "config": {"workload": "encrypted DB N=2^16 K=2^15 ell=%d n1=%d deg59 work level %d" % (c["ell"], c["n1"],
                                                                                                 ctx.work_level),
                   "storage_tier": db.info()["tier"], "db_bytes": db.info()["bytes"]},
        "form": "CUDA graph replay, inputs resident",
        "batched": {"queries": B, "ms_per_pass": ms_b, "value": B * K / (ms_b / 1000.0), "unit": UNIT},
        "plaintext_db": {"ms_per_step": ms_pt, "value": K / (ms_pt / 1000.0), "unit": UNIT},
        "mac_ct": {"ms": mac_ms, "launches": mac_n, "algorithmic_bytes": mac_b, "gbs": mac_gbs,
                   "frac": (mac_gbs / hbm) if mac_gbs else None, "peak_gbs": hbm, "peak": hbm_src},
        "stages_ms_eager": stages,
        "enroll_s_host": enroll_s, "load_s": load_s,
        "server_prerotation": {"load_s": load_tbs_s, "ms_per_step": ms_tbs, "value": K / (ms_tbs / 1000.0),
                               "unit": UNIT, "membership_abs_err": err_tbs},
        "membership_abs_err": err, "clocks": clocks,
    }
    return line


def run_sharded(args):
    """Block-sharded match across the ranks, one GPU each: the K=2^20 identification database
    (32 groups of 2^15 templates) split along group boundaries (shard.template_shard), the query
    broadcast once, every rank matching its groups (identification, templates encoded per query
    unless --identify-tier says otherwise) and rank 0 receiving the per-group ciphertexts with
    point-to-point tensor transfers and reducing them (fr_membership_reduce: mod-q sum, then
    RotateAndSum) into one membership ciphertext. The total work is fixed, so the scaling is
    strong: value = K / (max over ranks of the step time)."""
    import torch

    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import shard
    from paper_2604_00546_gb300 import workloads as W

    ws, rank, local = dist_env()
    D = None
    if ws > 1:
        import torch.distributed as D
        D.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(device=torch.device("cuda", local))
    cfg = "identify"
    c = W.CONFIGS[cfg]
    T, q, planted = W.workload(cfg)
    K = len(T)
    slots = 1 << (c["log_n"] - 1)
    Ts, (g0, g1) = shard.template_shard(T, slots, ws, rank)
    ctx = fr.Context(device=local, cuda_stream=stream.cuda_stream, db_tier=args.identify_tier,
                     **W.ctx_params(cfg, level_mode=args.level_mode), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum,
                     hoist_giants=args.hoist_giants,
                     hoist_babies=args.hoist_babies)
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(cfg))
    ctx.load_keys(keys)
    db = ctx.load_db(Ts) if g1 > g0 else None
    query = shard.share_query(ctx, ctx.encrypt(keys, q, W.enc_seed(cfg)) if rank == 0 else None, D)
    query.upload()
    mode = fr.FR_MODE_MEMBERSHIP

    def step():
        return shard.sharded_match(ctx, db, query, mode, D)

    for _ in range(max(1, args.warmup)):
        res = step()
    got = float(ctx.decrypt(keys, res[0])[0]) if rank == 0 else None
    del res
    steps = max(1, args.steps // 3)
    sampler = ClockSampler(local)
    sampler.start()
    if D:
        D.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        res = step()
        ctx.sync()
    torch.cuda.synchronize()
    ms = 1000.0 * (time.perf_counter() - t0) / steps
    clocks = sampler.stop()
    tmax = max_over_ranks(ms, D, torch.device("cuda", local) if D and D.get_backend() == "nccl" else None)
    if rank == 0:
        from numpy.polynomial import chebyshev as npc
        s = T.astype(np.float64) @ q
        sp = np.zeros(((K + slots - 1) // slots) * slots)
        sp[:K] = s
        pref = float(npc.chebval(sp, fr.cheb_coeffs(c["cheb_degree"], c["threshold"])).sum())
        line = {
            "metric": "block-sharded membership: templates matched/s over all ranks (K=2^20, 32 groups)",
            "value": K / (tmax / 1000.0), "unit": UNIT, "n_gpus": ws, "steps": steps, "ms_per_step": tmax,
            "higher_is_better": True, "scaling": "strong", "dtype": "u64",
            "data": "synthetic (seeded Gaussian L2-normalised templates, 32 planted duplicates at cosine 0.8)",
            "config": {"workload": "membership N=2^16 K=2^20 ell=512 deg59, groups split across ranks",
                       "groups": -(-K // slots), "groups_rank0": g1 - g0, "tier": db.info()["tier"] if db else None,
                       "parallelism": f"block-sharded x{ws}",
                       "timing": "host wall clock around each step with the device synchronised, max over ranks"},
            "check": {"membership_decrypted": got, "membership_fp64": pref, "abs_err": abs(got - pref)},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if D:
        D.barrier()
        D.destroy_process_group()


def run_tensor_probe(args):
    """The tensor-core question of an exact NTT: the measured dense INT8 rate of this GPU (cuBLAS
    through torch._int_mm, 8192^3, int8 x int8 -> int32) beside the bf16 rate, and the rate an
    exact tensor-core NTT would need to beat the CUDA-core NTT measured here. An exact product of
    residues below 2^60 split into 8-bit limbs takes 64 int8 multiply-adds; a 2^16-point NTT as
    two dense 256-point DFT passes (four-step form) takes 2 x 2^16 x 256 modular products per
    polynomial, so 2 x 2^16 x 256 x 64 x 2 int8 operations, against the CUDA-core transform's
    measured microseconds per polynomial (fr_ntt_time, 1024 polynomials)."""
    import torch

    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = 8192

    def rate(fn, flops):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 1e30
        for _ in range(10):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return flops / (best / 1000.0)

    a8 = torch.randint(-128, 127, (n, n), dtype=torch.int8, device=dev)
    b8 = torch.randint(-128, 127, (n, n), dtype=torch.int8, device=dev)
    int8_ops = rate(lambda: torch._int_mm(a8, b8), 2.0 * n ** 3)
    a16 = torch.randn(n, n, dtype=torch.bfloat16, device=dev)
    b16 = torch.randn(n, n, dtype=torch.bfloat16, device=dev)
    bf16_flops = rate(lambda: a16 @ b16, 2.0 * n ** 3)
    ctx = fr.Context(device=local, **W.ctx_params("membership", level_mode=1))
    npol = 1024
    f_us, i_us = ctx.ntt_time(npol, ctx.work_level, 5)
    per_poly_s = 0.5 * (f_us + i_us) * 1e-6 / npol
    ops_per_poly = 2.0 * (1 << 16) * 256 * 64 * 2
    line = {
        "metric": "tensor-core question of the exact NTT", "int8_dense_ops_per_s": int8_ops,
        "bf16_dense_flops_per_s": bf16_flops, "int8_over_bf16": int8_ops / bf16_flops,
        "cuda_core_ntt_us_per_poly": per_poly_s * 1e6, "int8_ops_per_poly_dense_dft": ops_per_poly,
        "int8_ops_per_s_needed_to_match": ops_per_poly / per_poly_s,
        "int8_time_per_poly_us_at_measured_rate": ops_per_poly / int8_ops * 1e6,
        "verdict": "tensor cores slower" if ops_per_poly / int8_ops > per_poly_s else "tensor cores faster",
    }
    return line


def run_mac_small(args):
    """The batched diagonal MAC on a small case, for profiling: N = 2^13, Q = 60 + 4 x 45, P = 3 x 60,
    ell = 512, n1 = 32 (the headline's BSGS split), baby steps in Q_l u P, 4096 seeded templates,
    4 queries per fr_match_batch (scores). About 2 GB on the device; the diagonals (268 MB) are
    twice the L2. Returns the batch time."""
    import torch

    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import workloads as W
    cfg = dict(log_n=13, q_bits=[60] + [45] * 4, p_bits=[60, 60, 60], dnum=2, scale_bits=45, ell=512, n1=32,
               cheb_degree=0, threshold=0.5)
    ctx = fr.Context(device=0, hoist_babies=1, **cfg)
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_SCORES), 0x5EED0A11)
    ctx.load_keys(keys)
    db = ctx.load_db(W.templates(4096, cfg["ell"], 21))
    rng = np.random.default_rng(1)
    qs = []
    for i in range(4):
        q = rng.standard_normal(cfg["ell"])
        qs.append(ctx.encrypt(keys, q / np.linalg.norm(q), 900 + i))
    ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = ctx.match_batch(db, qs, fr.FR_MODE_SCORES)
        ctx.sync()
        ms.append(1000.0 * (time.perf_counter() - t0))
    free, total = torch.cuda.mem_get_info(0)
    return {"mode": "mac-small", "queries": len(qs), "outputs": len(outs), "batch_ms": ms,
            "device_gb": (total - free) / 1e9}


def run_ntt_sweep(args):
    """The batched NTT alone (fr_ntt_time) at the headline ring (N = 2^16, working level 8,
    shapes picked by the tuner): microseconds per forward and inverse launch sequence and
    butterflies per second against the register-only butterfly rate, per batch size. With one
    size it is also the small case the NTT's ncu captures run on."""
    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import workloads as W

    ws, rank, local = dist_env()
    ctx = fr.Context(device=local, **W.ctx_params("membership", level_mode=1))
    peak = fr.butterfly_peak(local)
    rows = []
    for n in args.ntt_sizes:
        f, i = ctx.ntt_time(n, ctx.work_level, 5)
        bf = n * (1 << 15) * 16.0
        rows.append({"polys": n, "fwd_us": f, "inv_us": i, "fwd_frac": bf / (f * 1e-6) / peak,
                     "inv_frac": bf / (i * 1e-6) / peak})
    return {"metric": "batched NTT, N=2^16: time per launch sequence and fraction of the butterfly peak",
            "butterfly_peak_per_s": peak, "shapes": ctx.ntt_tuning(), "rows": rows}


def run_reference(args):
    """Reference arm: the CPU oracle (the paper has no runnable code) on the same workload,
    metric and unit. Each step is one whole membership query of the oracle on the host cores;
    the oracle needs no warm-up (no caches or code generation), so none is run, and the
    number of timed queries is capped so that the run ends within a few minutes. Under
    torchrun only rank 0 works; the other ranks exit at once."""
    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return
    from paper_2604_00546_gb300 import workloads as W
    cfg = args.config
    T, q, _ = W.workload(cfg)
    lq = W.work_level(cfg, args.level_mode)
    t_all = time.perf_counter()
    secs, cores, _ = oracle_queries(cfg, T, q, W.key_seed(cfg), W.enc_seed(cfg), lq, budget_s=100.0,
                                    max_queries=max(1, args.steps), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum,
                                    hoist=bool(args.hoist_giants), babies_pq=bool(args.hoist_babies))
    wall = time.perf_counter() - t_all
    per = float(np.mean(secs))
    value = len(T) / per
    sample = (f"{len(secs)} whole membership queries of the oracle (K={len(T)}, working level {lq}), "
              f"{', '.join('%.1f s' % x for x in secs)}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(secs), "steps_requested": args.steps, "warmup": 0, "warmup_requested": args.warmup,
        "ms_per_step": 1000.0 * per, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic (seeded Gaussian L2-normalised templates, 32 planted duplicates at cosine 0.8)",
        "config": {"workload": "membership N=2^16 K=2^15 ell=512 n1=32 deg59", "K": len(T), "log_n": 16,
                   "work_level": lq},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "timed_s": float(np.sum(secs)), "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


# Kernel-time share of each region class in one headline membership match, and the NTT passes'
# DRAM bytes (read + written) per algorithmic byte, from the committed one-pass launch list of
# that match (ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
# --cache-control none; see profiles/launches_membership_N65536_K32768_level8.md). Valid only for
# the CUDA sources whose combined SHA-256 (csrc_sha256) is listed: then the regions of the bench
# line are these shares of the timed step; otherwise they come from the profiled replays and the
# NTT traffic is null.
LAUNCH_LIST = {
    "sha256": ["606e3b6d14d6bb44f1e83024d1b3c935de61ae6aaaca7c70ba7160ac288a57b5"],
    "share": {"ntt": 0.5483, "mac": 0.1334, "ip": 0.1237, "modup": 0.0553, "moddown": 0.0541, "rescale": 0.0511,
              "tensor": 0.0334, "misc": 0.0008, "copy": 0.0},
    "ntt_dram_per_alg_byte": 1.760,
    "keyswitch_dram_gbs": 2948.4,
}

# kernel name prefix -> region class, for reading a launch list
KERNEL_CLASS = (("k_ntt", "ntt"), ("k_modup", "modup"), ("k_ip", "ip"), ("k_baby0_pq", "ip"), ("k_p2q", "moddown"),
                ("k_moddown", "moddown"), ("k_rs_", "rescale"), ("k_rescale", "rescale"), ("k_leaf_lift", "rescale"),
                ("k_tensor", "tensor"), ("k_mac", "mac"))


def csrc_sha256():
    """SHA-256 over the package's CUDA sources (names and contents, in name order)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2604_00546_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


# the configuration the launch list was taken on: the headline membership match with the bench's
# defaults (set by run_ours from its arguments)
LAUNCH_LIST_CONFIG = {"ell": 512, "level_mode": 1, "sum_radix": 8, "hoist_giants": 1, "hoist_babies": 1, "hoist_sum": 1}
_RUN_CONFIG = {}


def launch_list_valid():
    """True when the committed launch list describes this run: the same CUDA sources and the
    headline configuration."""
    return (bool(LAUNCH_LIST["share"]) and csrc_sha256() in LAUNCH_LIST["sha256"]
            and _RUN_CONFIG == LAUNCH_LIST_CONFIG)


def keyswitch_entry(regions, hbm_peak, hbm_kind):
    """Aggregate rate of the key switches' memory-bound kernels (ModUp base conversion, inner
    products, ModDown base conversion): their algorithmic bytes over their time in the step, and,
    from the committed launch list when it matches the sources, the DRAM bytes those kernels
    moved over their durations. Their NTTs are arithmetic-bound and counted with the NTT."""
    parts = ("modup", "ip", "moddown")
    ms = sum(regions[r]["ms"] for r in parts)
    by = sum(regions[r]["bytes"] for r in parts)
    gbs = by / (ms / 1000.0) / 1e9 if ms > 0 else 0.0
    e = {"kernels": "k_modup, k_ip, k_ip_sum, k_baby0_pq, k_p2q", "ms_per_step": ms, "algorithmic_bytes": by,
         "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak, "peak_kind": hbm_kind,
         "dram_view": None}
    if launch_list_valid() and LAUNCH_LIST.get("keyswitch_dram_gbs"):
        g = LAUNCH_LIST["keyswitch_dram_gbs"]
        e["dram_view"] = {"achieved": g, "frac": g / hbm_peak,
                          "source": "DRAM bytes / durations of those launches in the committed launch list"}
    return e


def roofline(regions, log_n, device, fr):
    """Roofline entry of the region with the largest device time.

    The NTT is bound by 64-bit modular arithmetic, not by HBM: its working set per launch
    sits in L2 and the per-element work is log2(N)/2 butterflies. It is reported against
    the butterfly rate of the same arithmetic with operands in registers, measured on this
    GPU by the library (fr_butterfly_peak). The other regions stream keys and diagonals
    from HBM and are reported against the measured copy bandwidth."""
    dom = max(regions, key=lambda r: regions[r]["ms"])
    d = regions[dom]
    secs = d["ms"] / 1000.0
    nl = max(1, d["launches"])
    hbm_peak, hbm_kind = load_peaks()
    gbs = d["bytes"] / secs / 1e9 if secs > 0 else 0.0
    roof = {"kernel": dom, "launches": d["launches"], "avg_launch_us": 1e6 * secs / nl,
            "bytes_per_launch": d["bytes"] / nl}
    if dom == "ntt":
        bfly = d["bytes"] / 16.0 * (log_n / 2.0)   # 16 B per element (read + write) -> log2(N)/2 butterflies
        peak = fr.butterfly_peak(device) / 1e9
        achieved = bfly / secs / 1e9 if secs > 0 else 0.0
        traffic = None
        if LAUNCH_LIST["ntt_dram_per_alg_byte"] and launch_list_valid():
            traffic = LAUNCH_LIST["ntt_dram_per_alg_byte"] * d["bytes"] / nl
        roof.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gbutterfly/s",
                     "frac": achieved / peak if peak > 0 else None,
                     "peak_kind": "measured: register-only butterfly loop on this GPU (fr_butterfly_peak)",
                     "butterflies_per_launch": bfly / nl, "traffic": traffic,
                     "hbm_view": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                                  "peak_kind": hbm_kind}})
    else:
        roof.update({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                     "peak_kind": hbm_kind, "traffic": None})
    return roof


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2604_00546_gb300 import fr
    from paper_2604_00546_gb300 import workloads as W

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    cfg = args.config
    if args.ell:   # a smaller template dimension (profiling cases); the headline is ell = 512
        cfg = dict(W.CONFIGS[cfg], ell=args.ell)
    c = W.CONFIGS[cfg] if isinstance(cfg, str) else cfg
    mode = c["mode"]
    _RUN_CONFIG.clear()
    if args.config == "membership":
        _RUN_CONFIG.update({"ell": c["ell"], "level_mode": args.level_mode, "sum_radix": args.sum_radix,
                            "hoist_giants": args.hoist_giants, "hoist_babies": args.hoist_babies,
                            "hoist_sum": args.hoist_sum})
    T, q, planted = W.workload(cfg)
    K = len(T)
    t0 = time.perf_counter()
    ctx = fr.Context(device=local, cuda_stream=stream.cuda_stream, **W.ctx_params(cfg, level_mode=args.level_mode), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum, hoist_giants=args.hoist_giants,
                     hoist_babies=args.hoist_babies)
    rots = ctx.required_rotations(mode)
    keys = ctx.keygen(rots, W.key_seed(cfg))
    t_keygen = time.perf_counter() - t0
    ctx.load_keys(keys)
    db = ctx.load_db(T)
    host_q = ctx.encrypt(keys, q, W.enc_seed(cfg))
    dev_q = ctx.encrypt(keys, q, W.enc_seed(cfg)).upload()
    ctx.sync()
    t_setup = time.perf_counter() - t0
    lq = ctx.work_level

    def step(cx, d, query):
        return cx.match(d, query, mode)

    for _ in range(args.warmup):
        out = step(ctx, db, dev_q)
    ctx.sync()
    # correctness of the last warm-up output (decrypted membership value vs FP64)
    from numpy.polynomial import chebyshev as npc
    s = T.astype(np.float64) @ q
    n = 1 << (c["log_n"] - 1)
    G = (K + n - 1) // n
    sp = np.zeros(G * n)
    sp[:K] = s
    pref = npc.chebval(sp, fr.cheb_coeffs(c["cheb_degree"], c["threshold"])).sum()
    got = float(ctx.decrypt(keys, out[0])[0])
    out_words = out[0].export() if (rank == 0 and ws == 1 and not args.no_cpu_baseline) else None
    del out

    sampler = ClockSampler(local)
    lat = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    n_launch0 = ctx.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    outs = []
    for i in range(args.steps):
        outs.append(step(ctx, db, dev_q))
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    n_launch = ctx.launch_count() - n_launch0
    clocks = sampler.stop()
    for i in range(args.steps):
        lat.append(ev[i].elapsed_time(ev[i + 1]))
    total_ms = ev[0].elapsed_time(ev[-1])
    del outs
    tmax = max_over_ranks(total_ms, dist, dev)
    value = whole_job_value(ws, K * args.steps, tmax)

    # per-region device time: the same steps again as profiled graph replays (the match
    # captured with CUDA events around the timed regions as graph nodes, replayed once per
    # step). One region class per replay (fr_profile_only), so only that class's launches carry
    # event records and every other launch runs as in the timed steps.
    nprof = 3
    regions, prof_match = {}, {}
    for r in REGIONS + ("stage:",):
        ctx.profile_only(r)
        ctx.profile(True)
        for i in range(nprof):
            outs = step(ctx, db, dev_q)
        torch.cuda.synchronize()
        if r == "stage:":
            stages = {st: ctx.profile_read("stage:" + st)[0] / nprof for st in STAGES}
        else:
            ms, nl, by = ctx.profile_read(r)
            regions[r] = {"ms": ms / nprof, "launches": nl / nprof, "bytes": by / nprof}
        prof_match[r] = ctx.profile_read("match")[0] / nprof
        ctx.profile(False)
        del outs
    ctx.profile_only("")
    # each class's replay carries event records around that class's launches only, and each
    # record adds latency to its region: these times are upper bounds. When the committed launch
    # list matches the sources, the regions are its kernel-time shares of the timed step.
    replayed = {r: dict(v) for r, v in regions.items()}
    regions_source = "profiled replays, one region class each (upper bounds: event latency inside)"
    if launch_list_valid():
        for r in regions:
            regions[r]["ms"] = LAUNCH_LIST["share"].get(r, 0.0) * (tmax / args.steps)
        regions_source = ("kernel-time shares of the committed one-pass launch list (ncu, current sources) x the "
                          "timed step")

    # end to end through the C ABI: host query -> H2D (the working-level limbs) -> match -> D2H
    h2d = 2 * (lq + 1) * (1 << c["log_n"]) * 8
    e2e_t = []
    d2h = 0
    for i in range(max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        a = time.perf_counter()
        res = step(ctx, db, host_q)
        words = [r.export() for r in res]
        e2e_t.append(time.perf_counter() - a)
        d2h = sum(w.nbytes for w in words)
    e2e_value = whole_job_value(ws, K, 1000.0 * max_over_ranks(float(np.mean(e2e_t)), dist, dev))

    # the plain per-query form: the same fr_match with every kernel launched per call (no graph)
    ctx.use_graphs(False)
    for _ in range(2):
        out = step(ctx, db, dev_q)
    got_p = float(ctx.decrypt(keys, out[0])[0])
    del out
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    npl = max(3, args.steps // 2)
    torch.cuda.synchronize()
    e0.record(stream)
    outs = [step(ctx, db, dev_q) for _ in range(npl)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1) / npl
    del outs
    ctx.use_graphs(True)
    plain = {"form": "one query per fr_match, kernels launched per call (no CUDA graph)", "ms_per_step": ms_p,
             "value": K / (ms_p / 1000.0), "unit": UNIT, "membership_abs_err": abs(got_p - pref)}

    # batched launches: B distinct queries per pass (fr_match_batch), same database
    batched = None
    if args.batch > 1:
        qs = [ctx.encrypt(keys, q, W.enc_seed(cfg, r)).upload() for r in range(args.batch)]
        for _ in range(2):
            outb = ctx.match_batch(db, qs, mode)
        ctx.sync()
        got_b = [float(ctx.decrypt(keys, o[0])[0]) for o in outb]
        del outb
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nb = max(3, args.steps // 2)
        torch.cuda.synchronize()
        e0.record(stream)
        outs = [ctx.match_batch(db, qs, mode) for _ in range(nb)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1) / nb
        del outs
        # profiled replays of the batch, one for the stages and one for every region: where
        # its time goes
        b_replay = {}
        for only in ("stage:", ""):
            ctx.profile_only(only)
            ctx.profile(True)
            outs = ctx.match_batch(db, qs, mode)
            torch.cuda.synchronize()
            if only:
                b_stages = {st: ctx.profile_read("stage:" + st)[0] for st in STAGES}
            else:
                b_regions = {r: ctx.profile_read(r)[0] for r in REGIONS}
            b_replay[only or "all regions"] = ctx.profile_read("match")[0]
            ctx.profile(False)
            del outs
        ctx.profile_only("")
        batched = {"queries": args.batch, "ms_per_batch": ms_b, "value": args.batch * K / (ms_b / 1000.0),
                   "unit": UNIT, "max_abs_err": max(abs(v - pref) for v in got_b),
                   "vs_plain_per_query": ms_p / (ms_b / args.batch),
                   "profiled_replay_ms": b_replay, "stages_ms": b_stages, "regions_ms": b_regions}

    # the same query on the whole modulus chain (no level drop), for comparison
    full = None
    if args.level_mode == 1 and not args.no_full_chain and lq < len(c["q_bits"]) - 1:
        ctx_f = fr.Context(device=local, cuda_stream=stream.cuda_stream, **W.ctx_params(cfg, level_mode=0), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum, hoist_giants=args.hoist_giants,
                     hoist_babies=args.hoist_babies)
        ctx_f.load_keys(keys)
        db_f = ctx_f.load_db(T)
        dq_f = ctx_f.encrypt(keys, q, W.enc_seed(cfg)).upload()
        for _ in range(2):
            out = step(ctx_f, db_f, dq_f)
        ctx_f.sync()
        got_f = float(ctx_f.decrypt(keys, out[0])[0])
        del out
        nf = max(3, args.steps // 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        outs = [step(ctx_f, db_f, dq_f) for _ in range(nf)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms_f = e0.elapsed_time(e1) / nf
        del outs
        full = {"work_level": len(c["q_bits"]) - 1, "ms_per_step": ms_f, "value": K / (ms_f / 1000.0),
                "steps": nf, "membership_decrypted": got_f}
        del db_f, ctx_f

    # the same query by the rotated-query table of Algorithm 1 (schedule 1), for comparison
    table = None
    if not args.no_table:
        ctx_t = fr.Context(device=local, cuda_stream=stream.cuda_stream, schedule=1,
                           **W.ctx_params(cfg, level_mode=args.level_mode), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum, hoist_giants=args.hoist_giants,
                     hoist_babies=args.hoist_babies)
        ctx_t.load_keys(keys)
        db_t = ctx_t.load_db(T)
        dq_t = ctx_t.encrypt(keys, q, W.enc_seed(cfg)).upload()
        for _ in range(2):
            out = step(ctx_t, db_t, dq_t)
        ctx_t.sync()
        got_t = float(ctx_t.decrypt(keys, out[0])[0])
        del out
        nt = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        outs = [step(ctx_t, db_t, dq_t) for _ in range(nt)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms_t = e0.elapsed_time(e1) / nt
        del outs
        table = {"schedule": "table (Algorithm 1)", "ms_per_step": ms_t, "value": K / (ms_t / 1000.0), "steps": nt,
                 "rotations": fr.rotation_count(c["ell"], c["n1"], G, 1),
                 "rotations_on_demand": fr.rotation_count(c["ell"], c["n1"], G, 0),
                 "membership_abs_err": abs(got_t - pref)}
        del db_t, ctx_t

    # the hybrid comparator (Chebyshev sign interpolant, then (1 + f_4) / 2; 4 more levels) on
    # the same query: its membership value is the count of the planted matches
    hybrid = None
    if not args.no_hybrid:
        ctx_h = fr.Context(device=local, cuda_stream=stream.cuda_stream, comparator=1,
                           **W.ctx_params(cfg, level_mode=args.level_mode), sum_radix=args.sum_radix, hoist_sum=args.hoist_sum,
                           hoist_giants=args.hoist_giants,
                     hoist_babies=args.hoist_babies)
        ctx_h.load_keys(keys)
        db_h = ctx_h.load_db(T)
        dq_h = ctx_h.encrypt(keys, q, W.enc_seed(cfg)).upload()
        for _ in range(max(3, args.warmup)):
            out = step(ctx_h, db_h, dq_h)
        ctx_h.sync()
        got_h = float(ctx_h.decrypt(keys, out[0])[0])
        del out
        nh = max(3, args.steps // 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        outs = [step(ctx_h, db_h, dq_h) for _ in range(nh)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms_h = e0.elapsed_time(e1) / nh
        del outs
        hybrid = {"comparator": "hybrid: degree-59 sign interpolant, then (1 + f_4(y)) / 2",
                  "work_level": ctx_h.work_level, "ms_per_step": ms_h, "value": K / (ms_h / 1000.0), "steps": nh,
                  "membership_decrypted": got_h, "planted": int(len(planted)),
                  "count_abs_err": abs(got_h - len(planted)),
                  "plain_comparator_membership": got}
        del db_h, ctx_h

    # roofline of the dominant region (largest device time), before the secondary workloads
    roof = roofline(regions, c["log_n"], local, fr)
    achieved = regions[roof["kernel"]]["bytes"] / (regions[roof["kernel"]]["ms"] / 1000.0) / 1e9

    # the secondary workloads, each with its own clocks and accuracy check
    secondary = None
    if ws == 1 and not args.no_secondary:
        secondary = {}
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.serve_seconds, sub.batch = 6, 3, args.serve_seconds_secondary, 4
        for name, fn in (("identify", run_identify), ("encrypted_db", run_encrypted), ("serving", run_serving),
                         ("multi", run_multi)):
            t_sub = time.perf_counter()
            try:
                secondary[name] = fn(sub)
            except Exception as e:  # reported in the line; the headline stands on its own
                secondary[name] = {"error": repr(e)}
            secondary[name]["wall_s"] = time.perf_counter() - t_sub
            torch.cuda.empty_cache()


    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        secs, cores, (o_ct, o_lvl) = oracle_queries(cfg, T, q, W.key_seed(cfg), W.enc_seed(cfg), lq,
                                                    sum_radix=args.sum_radix, hoist_sum=args.hoist_sum, hoist=bool(args.hoist_giants),
                                                    babies_pq=bool(args.hoist_babies))
        cpu = {"value": K / float(np.mean(secs)), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "one whole membership query of the oracle, K=%d at working level %d: %.1f s" % (K, lq, secs[0]),
               "seconds_per_query": float(np.mean(secs)),
               "bit_exact_vs_gpu": bool(np.array_equal(o_ct, out_words)) if out_words is not None else None}

    if rank == 0:
        lat_sorted = sorted(lat)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded Gaussian L2-normalised templates, 32 planted duplicates at cosine 0.8)",
            "config": {"workload": "membership N=2^16 K=2^15 ell=%d n1=32 deg59" % c["ell"], "K": K, "log_n": c["log_n"],
                       "q_limbs": len(c["q_bits"]), "p_limbs": len(c["p_bits"]), "dnum": c["dnum"],
                       "work_level": lq, "level_mode": args.level_mode, "sum_radix": args.sum_radix,
                       "hoist_giants": args.hoist_giants, "hoist_babies": args.hoist_babies,
                       "hoist_sum": args.hoist_sum,
                       "parallelism": f"replicas x{ws}",
                       "l2": "working set (diagonals + evaluation keys, several GB) exceeds the 129 MB L2; no flush"},
            "latency_ms": {"p50": float(np.percentile(lat_sorted, 50)), "p99": float(np.percentile(lat_sorted, 99)),
                           "mean": float(np.mean(lat))},
            "hbm_gbs_dominant": achieved,
            "roofline": roof,
            "regions_ms_per_step": {r: regions[r]["ms"] for r in regions},
            "regions_sum_ms": sum(regions[r]["ms"] for r in regions),
            "regions_source": regions_source,
            "regions_replayed_ms": {r: replayed[r]["ms"] for r in replayed},
            "profiled_replay_ms": prof_match,
            "profiling": ("graph replays with CUDA events as graph nodes around one region class per replay "
                          "(fr_profile_only), %d replays per class; the Chebyshev branches run on one stream "
                          "in the region replays and on their two streams in the stage replays" % nprof),
            "regions_hbm_gbs": {r: (regions[r]["bytes"] / (regions[r]["ms"] / 1000.0) / 1e9 if regions[r]["ms"] > 0
                                    else 0.0) for r in regions},
            "stages_ms_per_step": stages,
            "keyswitch": keyswitch_entry(regions, *load_peaks()),
            "gpu_launches": int(n_launch),
            "ntt_autotune": ctx.ntt_tuning(),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "full_chain": full,
            "table_schedule": table,
            "plain_per_query": plain,
            "batched": batched,
            "hybrid_comparator": hybrid,
            "secondary": secondary,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "check": {"membership_decrypted": got, "membership_fp64": float(pref), "abs_err": abs(got - pref)},
            "setup_s": {"keygen": t_keygen, "total": t_setup},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="membership")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-full-chain", action="store_true")
    ap.add_argument("--no-table", action="store_true", help="skip the table-schedule comparison")
    ap.add_argument("--level-mode", type=int, default=1, choices=[0, 1])
    ap.add_argument("--hoist-babies", type=int, default=1, choices=[0, 1],
                    help="baby steps kept in Q_l u P with one ModDown per giant step (fr_params.hoist_babies)")
    ap.add_argument("--hoist-giants", type=int, default=1, choices=[0, 1],
                    help="giant steps of a (query, group) share one ModDown (0: one per rotation)")
    ap.add_argument("--sum-radix", type=int, default=8, choices=[2, 4, 8, 16, 32],
                    help="RotateAndSum radix of the membership result (2: one rotation per step)")
    ap.add_argument("--hoist-sum", type=int, default=1, choices=[0, 1],
                    help="the rotations of a RotateAndSum step share one ModDown (fr_params.hoist_sum)")
    ap.add_argument("--batch", type=int, default=8, help="queries per pass for the batched measurement (1: skip)")
    ap.add_argument("--serving", action="store_true", help="run the serving-loop workload instead")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-batch", type=int, default=8)
    ap.add_argument("--serve-slots", type=int, default=2)
    ap.add_argument("--identify", action="store_true", help="run the K=2^20 identification workload instead")
    ap.add_argument("--multi", action="store_true", help="run the 64-database batched workload instead")
    ap.add_argument("--multi-n", type=int, default=64)
    ap.add_argument("--multi-budget-gb", type=float, default=80.0, help="stored-diagonal budget of the plan")
    ap.add_argument("--identify-tier", type=int, default=2, choices=[0, 1, 2, 3])
    ap.add_argument("--encrypted-db", action="store_true",
                    help="run the encrypted-database membership workload instead")
    ap.add_argument("--db-ell", type=int, default=512, help="template dimension of --encrypted-db (512: the workload)")
    ap.add_argument("--no-hybrid", action="store_true", help="skip the hybrid-comparator comparison")
    ap.add_argument("--ntt-sweep", action="store_true", help="time the batched NTT alone per batch size instead")
    ap.add_argument("--ntt-sizes", type=int, nargs="+", default=[1, 4, 16, 30, 64, 128, 248, 512, 1024])
    ap.add_argument("--mac-small", action="store_true",
                    help="run the batched MAC on a small case (N = 2^13, 4 queries) instead, for profiling")
    ap.add_argument("--ell", type=int, default=0,
                    help="template dimension of the membership workload (0: 512); smaller cases for profiling")
    ap.add_argument("--tensor-probe", action="store_true",
                    help="measure the INT8 / bf16 tensor rates against the CUDA-core NTT instead")
    ap.add_argument("--shard", action="store_true",
                    help="run the block-sharded K=2^20 membership across the ranks instead (strong scaling)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary workloads (identification, encrypted database, serving, multi)")
    ap.add_argument("--serve-seconds-secondary", type=float, default=15.0,
                    help="length of the serving run inside the default bench line")
    args = ap.parse_args()
    if args.serving:
        print(json.dumps(run_serving(args)), flush=True)
    elif args.identify:
        print(json.dumps(run_identify(args)), flush=True)
    elif args.multi:
        print(json.dumps(run_multi(args)), flush=True)
    elif args.encrypted_db:
        print(json.dumps(run_encrypted(args)), flush=True)
    elif args.shard:
        run_sharded(args)
    elif args.tensor_probe:
        print(json.dumps(run_tensor_probe(args)), flush=True)
    elif args.ntt_sweep:
        print(json.dumps(run_ntt_sweep(args)), flush=True)
    elif args.mac_small:
        print(json.dumps(run_mac_small(args)), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
