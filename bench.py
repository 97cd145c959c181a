#!/usr/bin/env python
"""Benchmark of the joint P+B covariance path on GB300.

Default workload: cfg3_10bin (10 tomographic bins, 20 ell bins on [10, 5000],
N_chi = 256, N_M = 128, K = 32768, M = 181350).  Its covariance does not fit
as a dense square (263 GB), so one step is: device tables and exact counts
(cov_update), spectra and data vector (cov_spectra), and the whole joint
covariance with every term written once as a resident lower-packed matrix of
256 x 256 tiles (cov_assemble_band over all rows, 132 GB).  The metric is
unique covariance elements M(M+1)/2 per second.  The S/N stage (FP64
Cholesky of P, B and the joint vector) is timed in the same run on the 5-bin
workload, whose dense square fits (--snr-workload).

Workloads whose dense square fits (e.g. --workload cfg2_5bin) run the whole
path in one step, S/N included.  With --gpus N > 1 (torchrun) each rank runs
its own cosmology of a Fisher-style set (weak scaling, no collective on the
data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|split_bf16] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle arm
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "joint P+B covariance elements/s"
UNIT = "elements/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="cfg3_10bin")
    p.add_argument("--layout", default="auto", choices=["auto", "dense", "tiles"])
    p.add_argument("--snr-workload", default="cfg3_5bin",
                   help="dense workload of the S/N stage (its stored oracle S/N gives the error)")
    p.add_argument("--no-snr-10bin", action="store_true",
                   help="skip the default 10-bin joint S/N in place on packed tiles")
    p.add_argument("--no-snr-run", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--batch-bins", default="3,5,10:2",
                   help="tomographic bin counts of the batched Fisher run (n_t:n for the first n cosmologies only; "
                        "the 10-bin set-up takes ~23 s per cosmology, so the default times two of its 64)")
    p.add_argument("--snr-10bin", action="store_true",
                   help="also time the P and B cumulative S/N of the workload itself (besides the joint one), "
                        "in place on packed tiles, per --snr-rows")
    p.add_argument("--snr-rows", default="joint,B,P", help="row sets of --snr-10bin")
    p.add_argument("--snr-precision", default="auto", choices=["auto", "fp64", "split_bf16"],
                   help="covariance form of --snr-10bin (auto: the bench's own)")
    p.add_argument("--serve-requests", type=int, default=250)
    p.add_argument("--serve-rate", type=float, default=200.0)
    p.add_argument("--serve-budget-gb", type=float, default=160.0)
    p.add_argument("--serve-search", action="store_true",
                   help="binary search for the sustainable arrival rate on the same mix and seed")
    p.add_argument("--serve-search-requests", type=int, default=40)
    p.add_argument("--serve-slots", type=int, default=4)
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "split_bf16"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-form", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--model-a", action="store_true",
                   help="also run the concentration-scatter comparison (model A against model B)")
    p.add_argument("--model-a-workload", default="cfg3_5bin")
    p.add_argument("--model-a-nodes", type=int, default=8, help="concentration nodes of model A")
    p.add_argument("--no-pca", action="store_true", help="skip the principal components of the paper's set-up")
    p.add_argument("--no-coupling", action="store_true", help="skip the exact BB+PT couplings key")
    p.add_argument("--pca-bins", default="1,2", help="tomographic bin counts of the paper's set-up for the PCA key")
    p.add_argument("--chol-kernel", default="auto", choices=["auto", "tile"],
                   help="Cholesky trailing update: persistent (auto) or one CTA per 128 x 64 tile")
    p.add_argument("--paper-replica", action="store_true",
                   help="also run the S/N experiments of the paper's own set-up (Sec. 5)")
    return p.parse_args()


def rank_cosmology(fiducial, rank):
    """The cosmology one rank computes: rank 0 the fiducial, ranks 1-6 a +1% step
    of one parameter each, ranks 7-12 the -1% steps, then +-2%, and so on: every
    rank a different problem.  Ranks solve independent problems, so the data
    path has no collective (weak scaling)."""
    cosmo = dict(fiducial)
    if rank > 0:
        keys = ["Om", "sigma8", "h", "ns", "Ob", "w0"]
        i = rank - 1
        sign = 1.0 if (i // len(keys)) % 2 == 0 else -1.0
        cosmo[keys[i % len(keys)]] *= 1.0 + sign * 0.01 * (1 + i // (2 * len(keys)))
    return cosmo


def job_step_ms(ms, world, device):
    """The job's step time: the largest of the ranks' (all-reduce MAX when world > 1)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- CPU oracle
def oracle_run(name):
    from oracle.pipeline import OracleRun
    from paper_1812_07437_gb300 import workloads
    ntri = None
    path = os.path.join(ROOT, "tests", "golden", f"counts_{name}.txt")
    if os.path.exists(path):
        sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
        import make_counts
        ntri = make_counts.load(name)[1]
    t0 = time.perf_counter()
    r = OracleRun(workloads.get(name), ntri=ntri)
    return r, time.perf_counter() - t0


def oracle_elements(r, n, seed):
    """Seeded lower-triangle element pairs; half on the P/B diagonal blocks."""
    import numpy as np
    rng = np.random.default_rng(seed)
    a = rng.integers(0, r.M, n)
    b = rng.integers(0, r.M, n)
    return np.maximum(a, b), np.minimum(a, b)


def cpu_model():
    """The host CPU's model name and its core count (lscpu, else /proc/cpuinfo)."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                name = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu model")):
                    name = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return name or "unknown", os.cpu_count() or 1


_POOL_COV = None


def _pool_init(blob):
    import pickle
    global _POOL_COV
    _POOL_COV = pickle.loads(blob)


def _pool_work(job):
    """Per-element oracle sums over this worker's pairs from t_start for at
    most `seconds`; returns (elements done, seconds spent)."""
    a, b, t_start, seconds = job
    while time.time() < t_start:
        time.sleep(0.001)
    t0 = time.perf_counter()
    n = 0
    while n < len(a) and time.perf_counter() - t0 < seconds:
        _POOL_COV.element(int(a[n]), int(b[n]))
        n += 1
    return n, time.perf_counter() - t0


def oracle_rate(cov, a, b, seconds, workers):
    """Aggregate rate of the oracle's per-element sums on `workers` host
    processes (spawn: the parent may already hold a CUDA context), each on its
    own share of the seeded pairs, all started at the same moment."""
    import multiprocessing as mp
    import pickle
    blob = pickle.dumps(cov, protocol=5)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_pool_init, initargs=(blob,)) as pool:
        t_start = time.time() + 5.0
        jobs = [(a[k::workers], b[k::workers], t_start, seconds) for k in range(workers)]
        res = pool.map(_pool_work, jobs)
    n = sum(x[0] for x in res)
    rate = sum(x[0] / x[1] for x in res if x[1] > 0)
    return rate, n, max(x[1] for x in res)


def cpu_baseline(name, seconds):
    r, t_build = oracle_run(name)
    model, cores = cpu_model()
    a, b = oracle_elements(r, 8000000, 1234)
    rate, n, dt = oracle_rate(r.cov, a, b, seconds, cores)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": model,
            "sample": f"{n} of 8M seeded lower-triangle elements of {name} (M={r.M}), every term, per-element "
                      f"oracle sums for {dt:.1f} s on {cores} host processes ({model}); oracle "
                      f"tables/spectra build {t_build:.1f} s not included"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    r, t_build = oracle_run(args.workload)
    model, cores = cpu_model()
    seconds = 4.0  # per step: the oracle on every host core
    a, b = oracle_elements(r, 4000000, 4321)
    for _ in range(args.warmup):
        oracle_rate(r.cov, a, b, 1.0, cores)
    rates, ns = [], 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        rate, n, _ = oracle_rate(r.cov, a[k::args.steps], b[k::args.steps], seconds, cores)
        rates.append(rate)
        ns += n
    dt = time.perf_counter() - t0
    v = statistics.mean(rates)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "M": r.M, "sample_per_step": f"{seconds:.0f} s of elements"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": model,
                            "sample": f"{ns} seeded covariance elements of {args.workload} over {args.steps} "
                                      f"steps of {seconds:.0f} s on {cores} host processes; oracle build "
                                      f"{t_build:.1f} s not timed"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def stored_oracle_snr(name):
    """The oracle's cumulative S/N of a workload as stored by
    tests/golden/make_snr.py ({'P'|'B'|'J': [n_ell]}), or None (text only: no
    oracle code runs here)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"snr_{name}.txt")
    if not os.path.exists(path):
        return None
    out = {}
    for line in open(path):
        p = line.split()
        if p and not p[0].startswith("#"):
            out.setdefault(p[0], {})[int(p[1])] = float(p[2])
    return {k: np.array([v[c] for c in sorted(v)]) for k, v in out.items()}


def max_rel(a, b):
    import numpy as np
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    m = np.isfinite(a) & np.isfinite(b)
    return float(np.max(np.abs(a[m] / b[m] - 1.0))) if m.any() else None


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm
TILE = 256


def packed_tiles(M):
    nt = (M + TILE - 1) // TILE
    return nt * (nt + 1) // 2


# 2.75 GB per band at cfg3_10bin: 16 bands of 8.3 GB copied to larger pinned
# buffers measured 30% slower end to end
E2E_BANDS = 48


def band_cuts(M, n_chunks):
    """Tile-row boundaries giving bands of roughly equal tile counts."""
    import math
    nt = (M + TILE - 1) // TILE
    total = nt * (nt + 1) // 2
    cuts = [0]
    for k in range(1, n_chunks):
        t = int(math.sqrt(2.0 * k * total / n_chunks))
        if t > cuts[-1]:
            cuts.append(min(t, nt))
    if cuts[-1] != nt:
        cuts.append(nt)
    return [min(t * TILE, M) for t in cuts]


def launches_per_step(which_sizes, n_tri, split, packed=False, n_sub=8):
    """Kernels of libwlcov launched by one step (memsets and copies not counted)."""
    tables = 11          # chi_max, los, growth_norm, amplitude, sigma, halo, profiles, edges, norms, kernels, sigw2
    counts = 3 if n_tri > 0 else 2   # row table, mode counts, triangle counts
    spectra = 5 if n_tri > 0 else 3  # P and B spectra, B and P projections, data vector
    if split:
        # trispectrum table (rows_prep, pair signatures, BF16 rows, contraction) + factor rows (rows_prep,
        # signatures, BF16 rows) + inverse counts; then the contraction, the per-element products and the
        # Gaussian diagonal blocks, once (dense) or once per sub-band (packed band call)
        assemble = 4 + 3 + 1 + (3 * n_sub if packed else 3)
    else:
        # FP64 trispectrum rows + product, FP64 factor rows, SSC rows, inverse counts, products, Gaussian
        # blocks, SSC product
        assemble = 2 + 1 + 1 + 1 + 1 + 1 + 1 + 1
    snr = 0
    for ms in which_sizes:
        nb = (ms + 63) // 64
        # pack, first panel (diagonal block, then the panel solve fused with the slicing), per further panel
        # two update launches (look-ahead) and the next panel's two kernels, the last update, the prefix sums
        snr += 1 + 2 + 4 * (nb - 1) + 1 + 1
    return tables + counts + spectra + assemble + snr


def timed(stream, fn, steps, h, world):
    import torch
    torch.cuda.synchronize()
    h.profile(True)
    h.stage_times()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(steps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    stages = h.stage_times()
    h.profile(False)
    return e0.elapsed_time(e1), stages, out


# DRAM bytes (read + write) per launch of the contraction, from an ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of a small case of the
# same kernel (profiles/), scaled to the workload by the tiles it computes.  A
# figure is valid only while the device code of the contraction's source file,
# its launch order and its tile constants are unchanged: their text is
# fingerprinted.
TRAFFIC = {
    # workload: (bytes per band call, fingerprint at capture); profiles/k_syrk_pair_cfg3_4bin.md
    "cfg3_4bin": (28.18e9, "f06215df88edc9d3"),
    "cfg3_10bin": (28.18e9 * 251695 / 1326, "f06215df88edc9d3"),  # scaled by tiles from cfg3_4bin
}


def kernel_fingerprint():
    import hashlib
    src = open(os.path.join(ROOT, "paper_1812_07437_gb300", "csrc", "syrk_tc.cu")).read()
    parts = [ln for ln in src.splitlines() if ln.startswith("#define TW_") or ln.startswith("#define PR_")]
    parts.append(src[:src.index("// ---------------------------------------------------------------- host side")])
    c = src.index("int wl_tile_order(")
    parts.append(src[c:src.index("\n}\n", c)])
    return hashlib.sha256("".join("".join(parts).split()).encode()).hexdigest()[:16]  # layout-insensitive


def measured_traffic(workload):
    ent = TRAFFIC.get(workload)
    return ent[0] if ent and kernel_fingerprint() == ent[1] else None


def contraction_roofline(stages, elements, K, prec, N, long_kernel, sm_mhz=None):
    """Roofline of the 1-halo (chi, M) contraction, the kernel the metric is
    built on.  achieved / frac count the method's work, 2 K' FLOP per unique
    element (K' = K + N_chi with the super-sample columns); the split form
    issues three BF16 products per FMA (hi hi + hi lo + lo hi), reported beside
    it as achieved_issued / frac_issued.  The peak is cuBLAS BF16 measured at
    the SM clock in peak_sm_mhz; the run's own median clock is sm_mhz, and
    frac_issued_at_run_clock rescales the peak to it."""
    syrk_ms, syrk_calls = stages["syrk_1h"]
    avg_ms = syrk_ms / max(syrk_calls, 1)
    flops = 2.0 * elements * K
    achieved = flops / (avg_ms / 1e3) / 1e12
    if prec == N.COV_FP64:
        return {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s", "frac": achieved / 1.25,
                "traffic": None, "kernel": "k_gemm_lower (FP64 1-halo contraction)", "launch_ms": avg_ms,
                "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak available)"}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    key = "bf16_tflops_sustained" if long_kernel else "bf16_tflops"
    peak = peaks[key]
    peak_mhz = (peaks.get("clocks_under_load") or {}).get("sm_mhz_median")
    issued = 3.0 * achieved
    out = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "frac_algorithmic": achieved / peak, "achieved_issued": issued, "frac_issued": issued / peak,
           "traffic": None,
           "kernel": "k_syrk_pair (tcgen05.mma.cta_group::2 split-BF16 1-halo + SSC contraction, 256x512 pair tiles)",
           "launch_ms": avg_ms, "sm_mhz": sm_mhz, "peak_sm_mhz": peak_mhz,
           "peak_source": f"MEASURED_PEAKS.json {key}, of measured"}
    if sm_mhz and peak_mhz:
        out["frac_issued_at_run_clock"] = issued / (peak * sm_mhz / peak_mhz)
    return out


def dense_run(h, wl, cosmo, prec, stream, steps, warmup, world, fp64_form, fp64_steps=2):
    """The whole path on a workload whose dense M x M square fits: tables,
    counts, spectra, the dense covariance and the three cumulative S/N
    (P, B, joint) by FP64 Cholesky."""
    import numpy as np
    import torch
    from paper_1812_07437_gb300 import native as N
    M = h.M
    dev = torch.device("cuda", torch.cuda.current_device())
    D = torch.zeros(M, dtype=torch.float64, device=dev)
    C = torch.zeros(M, M, dtype=torch.float64, device=dev)
    which = (N.COV_WHICH_P, N.COV_WHICH_B, N.COV_WHICH_JOINT)

    def step(p=prec):
        h.update(cosmo, stream)
        h.spectra(D, stream)
        h.assemble(C, N.COV_TERMS_ALL, p, stream)
        return [h.snr(C, D, w, stream) for w in which]

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
        ms, stages, snr = timed(stream, step, steps, h, world)
        out = {"ms_per_step": ms / steps, "stages": stages, "snr": snr, "D": D, "C": C}
        if fp64_form and prec != N.COV_FP64:
            if fp64_steps > 1:
                step(N.COV_FP64)
            ms64, st64, snr64 = timed(stream, lambda: step(N.COV_FP64), fp64_steps, h, 1)
            out["fp64"] = {"ms_per_step": ms64 / fp64_steps, "stages": st64, "snr": snr64}
            rel = max(float(np.nanmax(np.abs(a / b - 1))) for a, b in zip(snr, snr64))
            out["snr_rel_err_vs_fp64_form"] = rel
    return out


def serving_run(prec, n_req, rate, budget_gb, slots, device, seed=2024):
    """Continuous-batching serving loop (cov_server_*): a seeded Poisson stream
    of covariance + S/N requests of uneven size, each submitted at its arrival
    time; latency = arrival to S/N returned."""
    import numpy as np
    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300 import workloads
    from paper_1812_07437_gb300.server import Server
    reqs = workloads.serving_requests(n_req, rate, seed=seed)
    srv = Server(n_slots=slots, hbm_budget=int(budget_gb * 1e9), precision=prec, device=device)
    ids = []
    start = time.perf_counter()
    for t_arr, wl in reqs:
        dt = t_arr - (time.perf_counter() - start)
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(wl))
    infos = [srv.wait(i)[0] for i in ids]
    st = srv.stats()
    srv.close()
    done = [x for x in infos if x["state"] == N.COV_REQ_DONE]
    lat = np.array([x["t_done"] - x["t_submit"] for x in done]) if done else np.array([np.nan])
    wait = np.array([x["t_start"] - x["t_submit"] for x in done]) if done else np.array([np.nan])
    span = (max(x["t_done"] for x in done) - min(x["t_submit"] for x in infos)) if done else float("nan")
    el = sum(x["M"] * (x["M"] + 1) // 2 for x in done)
    return {"requests": n_req, "offered_rate_hz": rate, "completed": len(done),
            "rejected_never_fit": sum(1 for x in infos if x["state"] == N.COV_REQ_REJECTED),
            "failed": sum(1 for x in infos if x["state"] == N.COV_REQ_FAILED),
            "achieved_rate_hz": len(done) / span, "elements_per_s": el / span, "makespan_s": span,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_max_s": float(np.max(lat)), "queue_wait_p50_s": float(np.percentile(wait, 50)),
            "queue_wait_p90_s": float(np.percentile(wait, 90)),
            "M_served_max": max((x["M"] for x in done), default=0),
            "reused_resident": sum(x["reused"] for x in done), "max_running": st["max_running"],
            "peak_reserved_gb": st["peak_reserved"] / 1e9, "budget_gb": st["budget"] / 1e9, "slots": slots}


def serving_search(prec, n_req, budget_gb, slots, device, lo=0.05, hi=0.5, probes=4):
    """The highest arrival rate the server sustains on the serving mix (same
    seed): a rate is sustained when 90% of its requests start within 2 s of
    their arrival (the queue does not grow); bisection in log rate between lo
    and hi, each probe a fresh stream of n_req requests."""
    import math
    trials = []
    ok_rate = None
    for _ in range(probes):
        r = math.sqrt(lo * hi)
        sv = serving_run(prec, n_req, r, budget_gb, slots, device)
        good = sv["completed"] > 0 and sv["queue_wait_p90_s"] <= 2.0 and sv["failed"] == 0
        trials.append({"offered_rate_hz": r, "sustained": good, "achieved_rate_hz": sv["achieved_rate_hz"],
                       "queue_wait_p90_s": sv["queue_wait_p90_s"], "latency_p50_s": sv["latency_p50_s"],
                       "latency_p99_s": sv["latency_p99_s"], "completed": sv["completed"],
                       "rejected_never_fit": sv["rejected_never_fit"], "failed": sv["failed"],
                       "makespan_s": sv["makespan_s"]})
        if good:
            lo, ok_rate = r, r
        else:
            hi = r
    return {"sustainable_rate_hz": ok_rate, "criterion": "p90 queue wait <= 2 s", "requests_per_probe": n_req,
            "probes": trials}


def batch_run(prec, device, bins_list):
    """The batched Fisher set: 64 cosmologies (fiducial, +-1% and +-2% steps in
    six parameters, seeded draws within +-5%) for each tomographic bin count,
    16 ell bins, N_chi = 256, N_M = 128; one eager and tuned first cosmology,
    then graph replays.  For the smallest set-up the same 64 cosmologies also
    run through the plain calls, for the replay speed-up."""
    import numpy as np
    import torch
    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300 import workloads
    from paper_1812_07437_gb300.handle import Handle
    cos_all = workloads.fisher_cosmologies()
    dev = torch.device("cuda", device)
    out = {"cosmologies": len(cos_all), "ell_bins": 16, "n_chi": 256, "n_mass": 128}
    for k, ent in enumerate(bins_list):
        # "nt" runs every cosmology; "nt:n" the first n (a timing sample of a large set-up)
        nt, _, ncos = str(ent).partition(":")
        nt = int(nt)
        cos = cos_all[: int(ncos)] if ncos else cos_all
        wl = workloads.fisher_workload(nt)
        h = Handle(wl, device=device)
        st = torch.cuda.Stream(device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        snr, _, info = h.batch_snr(cos, precision=prec, tune=not ncos, stream=st)
        total = time.perf_counter() - t0
        el = h.M * (h.M + 1) // 2
        r = {"M": h.M, "total_s": total, "first_ms": info["first_ms"], "capture_ms": info["capture_ms"],
             "replay_ms_per_cosmology": info["replay_ms"], "single_graph_launch": bool(info["single_launch"]),
             "tuned": {"candidate": info["tuned"], "tc_kernel": info["tc_kernel"], "pr_group": info["pr_group"],
                       "chol_lookahead": info["chol_lookahead"], "chol_kernel": info["chol_kernel"],
                       "candidate_ms": info["candidate_ms"],
                       "candidates": ["pairs g8 look-ahead persistent", "pairs g4", "pairs g16", "one CTA per tile",
                                      "no look-ahead", "one-tile Cholesky update"]},
             "elements_per_s_replays": el / (info["replay_ms"] / 1e3), "snr_joint_fiducial": float(snr[0, 2, -1]),
             "cosmologies": len(cos)}
        if k == 0:
            D = torch.zeros(h.M, dtype=torch.float64, device=dev)
            C = torch.zeros(h.M, h.M, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            worst = 0.0
            with torch.cuda.stream(st):
                for j, c in enumerate(cos):
                    h.update(c, st)
                    h.spectra(D, st)
                    h.assemble(C, N.COV_TERMS_ALL, prec, st)
                    s3 = np.stack([h.snr(C, D, w, st) for w in (0, 1, 2)])
                    m = np.isfinite(s3)
                    worst = max(worst, float(np.max(np.abs(snr[j][m] / s3[m] - 1.0))))
            torch.cuda.synchronize()
            r["plain_ms_per_cosmology"] = (time.perf_counter() - t1) / len(cos) * 1e3
            r["max_rel_diff_vs_plain"] = worst
        out[f"{nt}bin"] = r
        h.close()
        torch.cuda.empty_cache()
    return out


def model_a_run(prec, device, name, n_conc):
    """Concentration scatter (model A, Eq. LogNormC, sigma_lnc = 0.18) against
    the median concentration (model B) on one workload: the whole dense step of
    each (tables, spectra, every covariance term, the three cumulative S/N),
    the contraction's roofline at n_conc times the halo-integral nodes, and the
    relative changes between the two models that Sec. 5.4 of the paper reports
    (data vector, covariance, S/N)."""
    import numpy as np
    import torch
    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300 import workloads
    from paper_1812_07437_gb300.handle import Handle
    dev = torch.device("cuda", device)
    res = {}
    for label, nc in (("model_B", 0), ("model_A", n_conc)):
        wl = workloads.get(name, bins=dict(n_conc=nc, sigma_lnc=workloads.SIGMA_LNC))
        h = Handle(wl, device=device)
        s = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s):
            r = dense_run(h, wl, dict(wl["cosmology"]), prec, s, 2, 1, 1, False)
        M = h.M
        elements = M * (M + 1) // 2
        K = wl["bins"]["n_chi"] * wl["bins"]["n_mass"] * max(1, nc)
        Kc = K + (wl["bins"]["n_chi"] if prec != N.COV_FP64 else 0)
        roof = contraction_roofline(r["stages"], elements, Kc, prec, N, long_kernel=True)
        res[label] = dict(r=r, nP=h.n_P, M=M, K=K, out={
            "K": K, "ms_per_full_step": r["ms_per_step"],
            # step time less the S/N stages (sequential on the stream); the assembly's own
            # stages overlap (the gather runs beside the contraction) and are not summed
            "assembly_elements_per_s": elements / ((r["ms_per_step"] - sum(
                v[0] for k, v in r["stages"].items() if k.startswith("snr")) / 2) / 1e3),
            "stages_ms_per_step": {k: v[0] / 2 for k, v in r["stages"].items() if v[1]},
            "contraction": {k: roof[k] for k in ("achieved", "peak", "unit", "frac", "launch_ms", "peak_source")
                            if k in roof},
            "snr_joint_max": float(np.nanmax(r["snr"][2]))})
        h.close()
    a, b = res["model_A"], res["model_B"]
    nP = a["nP"]
    dD = (a["r"]["D"] / b["r"]["D"] - 1.0).abs()
    var = (torch.diagonal(a["r"]["C"]) / torch.diagonal(b["r"]["C"]) - 1.0).abs()
    snr_rel = [float(np.nanmax(np.abs(np.asarray(x) / np.asarray(y) - 1.0)))
               for x, y in zip(a["r"]["snr"], b["r"]["snr"])]
    out = {"workload": name, "M": a["M"], "n_conc": n_conc, "sigma_lnc": workloads.SIGMA_LNC,
           "precision": "fp64" if prec == N.COV_FP64 else "split_bf16",
           "model_A": a["out"], "model_B": b["out"],
           "A_vs_B": {"D_P_max_rel": float(dD[:nP].max()), "D_B_max_rel": float(dD[nP:].max()),
                      "var_P_max_rel": float(var[:nP].max()), "var_B_max_rel": float(var[nP:].max()),
                      "snr_max_rel_P_B_joint": snr_rel}}
    del res
    torch.cuda.empty_cache()
    return out


def paper_run(device):
    """The paper's own set-up (its cosmology, 14 ell bins on [10, 5000], m_min = 1e9,
    Bullock median concentration, sigma_e = 0.3): the cumulative S/N at ell_max = 5000 of
    P, B and the joint vector for 1, 2 and 5 tomographic bins and of P for 10 bins, with
    the covariance term sets of the paper's Sec. 5 figures (G; G + NGins; G + NGssc; all),
    P at 10 bins also without shape noise, and the relative changes the paper states
    them by.  The covariances are assembled in the FP64 form: without photo-z scatter the
    tomographic kernels overlap strongly and the scaled covariance's smallest eigenvalue
    falls to ~1e-3 at 2 bins and below at 5, where the split form's ~1e-5 element error
    can move it below zero.  The 10-bin case holds the power-spectrum rows alone."""
    import numpy as np
    import torch
    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300 import workloads
    from paper_1812_07437_gb300.handle import Handle
    dev = torch.device("cuda", device)
    ins = N.COV_TERM_1H | N.COV_TERM_BBPT | N.COV_TERM_PB
    sets = {"G": N.COV_TERM_G, "G+NGins": N.COV_TERM_G | ins, "G+NGssc": N.COV_TERM_G | N.COV_TERM_SSC,
            "all": N.COV_TERMS_ALL}

    def last(v):
        v = np.asarray(v)
        f = v[np.isfinite(v)]
        return float(f[-1]) if f.size else None

    out = {}
    t0 = time.perf_counter()
    for nt, sigma_e, which in ((1, 0.3, "PBJ"), (2, 0.3, "PBJ"), (5, 0.3, "PBJ"), (10, 0.3, "P"), (10, 0.0, "P")):
        key = f"{nt}bin" + ("" if sigma_e > 0 else "_no_noise")
        wl = workloads.paper_workload(nt, sigma_e=sigma_e)
        joint = which == "PBJ"
        # 10 bins: a handle of the power-spectrum rows alone
        h = Handle(wl, device=device, rows=N.COV_ROWS_JOINT if joint else N.COV_ROWS_P)
        res = {"M": h.M, "n_P": h.n_P, "n_B": h.n_B}
        ws = (("P", N.COV_WHICH_P), ("B", N.COV_WHICH_B), ("joint", N.COV_WHICH_JOINT)) if joint else \
            (("P", N.COV_WHICH_P),)
        try:
            D = torch.zeros(h.M, dtype=torch.float64, device=dev)
            C = torch.zeros(h.M, h.M, dtype=torch.float64, device=dev)
            h.spectra(D)
            for name, terms in sets.items():
                h.assemble(C, terms, N.COV_FP64)
                res[name] = {w: last(h.snr(C, D, wi)) for w, wi in ws}
            del C, D
        except Exception as e:  # noqa: BLE001  (one case's failure is recorded; the others still run)
            res["error"] = f"{type(e).__name__}: {e}"
        out[key] = res
        h.close()
        torch.cuda.empty_cache()
    red = lambda a, b: 1.0 - a / b if a is not None and b is not None else None
    gain = lambda a, b: a / b - 1.0 if a is not None and b else None
    get = lambda key, s, w: out.get(key, {}).get(s, {}).get(w)
    out["derived"] = {
        "P_10bin_loss_vs_G": {k: red(get("10bin", k, "P"), get("10bin", "G", "P"))
                              for k in ("G+NGins", "G+NGssc", "all")},
        "P_loss_vs_10bin_all_terms": {f"{n}bin": red(get(f"{n}bin", "all", "P"), get("10bin", "all", "P"))
                                      for n in (5, 2, 1)},
        "B_loss_from_ssc": {f"{n}bin": red(get(f"{n}bin", "all", "B"), get(f"{n}bin", "G+NGins", "B"))
                            for n in (1, 2, 5)},
        "joint_loss_from_ssc": {f"{n}bin": red(get(f"{n}bin", "all", "joint"), get(f"{n}bin", "G+NGins", "joint"))
                                for n in (1, 2, 5)},
        "joint_gain_over_P": {f"{n}bin": gain(get(f"{n}bin", "all", "joint"), get(f"{n}bin", "all", "P"))
                              for n in (1, 2, 5)},
        "paper_states": {"P_10bin_loss_vs_G": {"G+NGins": 0.30, "G+NGssc": 0.40, "all": 0.45},
                         "P_loss_vs_10bin_all_terms": {"5bin": 0.01, "2bin": 0.05, "1bin": 0.25},
                         "B_loss_from_ssc": {"1bin": 0.20, "2bin": 0.15, "5bin": 0.15},
                         "joint_loss_from_ssc": {"1bin": 0.30, "2bin": 0.25, "5bin": 0.25},
                         "joint_gain_over_P": {"1bin": 0.10, "2bin": 0.10, "5bin": 0.10}}}
    out["seconds"] = time.perf_counter() - t0
    out["precision"] = "fp64"
    out["quadrature"] = "N_chi = 128, N_M = 96"
    return out


def pca_run(device, bins_list):
    """Principal components of the joint covariance (Sec. 6) of the paper's own
    set-up (its cosmology, 14 ell bins, Bullock median, replica quadrature),
    FP64 covariance (the set-up is too ill-conditioned for the split form):
    eigenvalues by one-sided Jacobi on the Cholesky factor, the per-mode S/N,
    and the modes needed for 90/95/99% of the total S/N (the paper: <~40% of
    the modes for 99% at 1 bin, <~20% at 2, <~10% at 5)."""
    import numpy as np
    import torch
    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300 import workloads
    from paper_1812_07437_gb300.handle import Handle
    dev = torch.device("cuda", device)
    out = {}
    for nt in bins_list:
        wl = workloads.paper_workload(nt)
        h = Handle(wl, device=device)
        D = torch.zeros(h.M, dtype=torch.float64, device=dev)
        C = torch.zeros(h.M, h.M, dtype=torch.float64, device=dev)
        h.spectra(D)
        h.assemble(C, N.COV_TERMS_ALL, N.COV_FP64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = h.pca(C, D)
        wall = time.perf_counter() - t0
        n = h.M
        flops = r["sweeps"] * 6.0 * n * n * (n - 1)  # per sweep: n(n-1)/2 pairs, 3 dot products + a rotation of 2n entries
        out[f"{nt}bin"] = {
            "M": n, "seconds": wall, "ms_cholesky": r["ms_cholesky"], "ms_jacobi": r["ms_jacobi"],
            "sweeps": r["sweeps"], "jacobi_fp64_tflops": flops / (r["ms_jacobi"] / 1e3) / 1e12,
            "eigenvalue_range": float(r["lam"][-1] / r["lam"][0]), "total_snr": float(np.sqrt(r["total_snr2"])),
            "modes_90_95_99": [r["modes_90"], r["modes_95"], r["modes_99"]],
            "fraction_for_99": r["modes_99"] / n}
        del C, D
        h.close()
        torch.cuda.empty_cache()
    out["paper_states_fraction_for_99"] = {"1bin": "<~0.40", "2bin": "<~0.20", "5bin": "<~0.10"}
    out["precision"] = "fp64 covariance, fp64 Jacobi"
    return out


def coupling_run(device, build_workload, snr_workload):
    """Exact bin-averaged BB+PT couplings (App. B, Eq. CovBB; COV_COUPLING_EXACT):
    the time to build them for a binning (cov_init with exact couplings minus
    cov_init without, on a coarse quadrature: they depend on the binning only),
    the spread of kappa N(l^b) (1 is the paper's 2 pi/(Omega l Delta l)), and the
    cumulative S/N at the largest ell bin of a workload (FP64 covariance) with
    the exact couplings against the paper's prefactor."""
    import numpy as np
    import torch
    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300 import workloads
    from paper_1812_07437_gb300.handle import Handle
    dev = torch.device("cuda", device)
    out = {}
    base = workloads.get(build_workload)
    wl = workloads.get(build_workload, bins=dict(base["bins"], n_chi=16, n_mass=12))
    walls = {}
    for name, cp in (("modes", N.COV_COUPLING_MODES), ("exact", N.COV_COUPLING_EXACT), ("exact2", N.COV_COUPLING_EXACT)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = Handle(wl, device=device, coupling=cp)
        walls[name] = time.perf_counter() - t0
        if name == "exact":
            ne, nt = h.counts()
            tris = []
            lo, hi, ncols = np.inf, -np.inf, []
            for A in range(h.n_ell):
                cols, G = h.coupling_gram(A)
                ncols.append(len(cols))
                if len(cols) == 0:
                    continue
                tris.append((A, cols, G))
            rd = h.row_desc()
            tri_bins = {}
            for r in rd[rd[:, 0] == 1]:
                tri_bins[int(r[7])] = tuple(int(x) for x in r[1:4])
            ntri_of = {b: int(nt[t]) for t, b in tri_bins.items()}
            # kappa N(A) = G N(A) / (N_tri N_tri') over every pair of columns of a
            # bin; column (Y, Z) of bin A belongs to the triangle sorted(A, Y, Z)
            for A, cols, G in tris:
                n = np.array([ntri_of[tuple(sorted((A, int(y), int(z))))] for y, z in cols], dtype=np.float64)
                kn = G.astype(np.float64) * float(ne[A]) / np.outer(n, n)
                lo, hi = min(lo, float(kn.min())), max(hi, float(kn.max()))
            out["kappa_N_range"] = [lo, hi]
            out["columns_per_bin"] = [min(ncols), max(ncols)]
        h.close()
    out["build_workload"] = build_workload
    out["build_s"] = min(walls["exact"], walls["exact2"]) - walls["modes"]
    res = {}
    for name, cp in (("modes", N.COV_COUPLING_MODES), ("exact", N.COV_COUPLING_EXACT)):
        h = Handle(workloads.get(snr_workload), device=device, coupling=cp)
        D = torch.zeros(h.M, dtype=torch.float64, device=dev)
        C = torch.zeros(h.M, h.M, dtype=torch.float64, device=dev)
        h.spectra(D)
        h.assemble(C, N.COV_TERMS_ALL, N.COV_FP64)
        res[name] = {w: float(h.snr(C, D, k)[-1]) for w, k in (("P", N.COV_WHICH_P), ("B", N.COV_WHICH_B),
                                                                 ("joint", N.COV_WHICH_JOINT))}
        del C, D
        h.close()
        torch.cuda.empty_cache()
    out["snr_workload"] = snr_workload
    out["snr_at_lmax"] = res
    out["snr_rel_change"] = {w: res["exact"][w] / res["modes"][w] - 1.0 for w in res["modes"]}
    out["precision"] = "fp64 covariance"
    return out


def snr_tiles_run(wl, prec, device, row_sets, chol=0):
    """Cumulative S/N of the workload's own data vector without a dense square:
    a handle in cumulative row order assembles its lower-packed tiles (plus one
    row for D) and cov_snr_tiles factorises them in place."""
    import numpy as np
    import torch
    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300.handle import Handle, packed_tiles
    dev = torch.device("cuda", device)
    out = {}
    for name, rows in row_sets:
        h = Handle(wl, device=device, rows=rows, order=N.COV_ORDER_CUMULATIVE, chol_kernel=chol)
        D = torch.zeros(h.M, dtype=torch.float64, device=dev)
        Ct = torch.empty(packed_tiles(h.M + 1) * 65536, dtype=torch.float64, device=dev)
        st = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(st):
            torch.cuda.synchronize()
            h.profile(True)
            h.stage_times()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(st)
            h.spectra(D, st)
            h.assemble_band(0, h.M, Ct, N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, prec, st)
            e1.record(st)
            snr = h.snr_tiles(Ct, D, st)
            e2.record(st)
            torch.cuda.synchronize()
            stg = h.stage_times()
            h.profile(False)
        chol_ms = stg["snr_cholesky"][0]
        out[name] = {"M": h.M, "assemble_ms": e0.elapsed_time(e1), "snr_ms": e1.elapsed_time(e2),
                     "cholesky_ms": chol_ms,
                     "cholesky_fp64_equivalent_tflops": h.M ** 3 / 3.0 / (chol_ms / 1e3) / 1e12,
                     "snr": [float(x) for x in snr], "snr_max": float(np.nanmax(snr))}
        del Ct, D
        h.close()
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300 import workloads
    from paper_1812_07437_gb300.handle import Handle

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    if args.precision == "auto":
        prec_name = "split_bf16" if os.environ.get("WLCOV_FORCE_FP64") is None and _has_split() else "fp64"
    else:
        prec_name = args.precision
    prec = N.COV_SPLIT_BF16 if prec_name == "split_bf16" else N.COV_FP64

    def rank_cosmo(wl):
        return rank_cosmology(wl["cosmology"], rank)

    wl = workloads.get(args.workload)
    cosmo = rank_cosmo(wl)
    wl = workloads.get(args.workload, cosmology=cosmo)
    chol = N.COV_CHOL_TILE if args.chol_kernel == "tile" else N.COV_CHOL_AUTO
    h = Handle(wl, device=local, chol_kernel=chol)
    M = h.M
    elements = M * (M + 1) // 2
    K = wl["bins"]["n_chi"] * wl["bins"]["n_mass"] * max(1, wl["bins"].get("n_conc", 0))
    Kc = K + (wl["bins"]["n_chi"] if prec != N.COV_FP64 else 0)  # SSC rows ride in the split contraction
    stream = torch.cuda.Stream(device=dev)
    packed = args.layout == "tiles" or (args.layout == "auto" and M * M * 8 > 64e9)
    gpu_index = int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[0]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    clk = ClockSampler(gpu_index)

    extra = {}
    if packed:
        # a1-a15: tables, counts, spectra and the whole lower-packed covariance
        # (256 x 256 tiles, resident in HBM), one band call covering every row
        D = torch.zeros(M, dtype=torch.float64, device=dev)
        Ct = torch.empty(packed_tiles(M) * TILE * TILE, dtype=torch.float64, device=dev)

        def step():
            h.update(cosmo, stream)
            h.spectra(D, stream)
            h.assemble_band(0, M, Ct, N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, prec, stream)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
            clk.start()
            time.sleep(0.4)
            ms_total, stages, _ = timed(stream, step, args.steps, h, world)
            clocks = clk.stop()
            # e2e through the public API: the covariance streamed to the host in
            # bands of about equal size, band k+1 computed while band k is copied
            cuts = band_cuts(M, E2E_BANDS)
            bands = list(zip(cuts[:-1], cuts[1:]))
            nmax = max(packed_tiles(b) - packed_tiles(a) for a, b in bands) * TILE * TILE
            dbuf = [torch.empty(nmax, dtype=torch.float64, device=dev) for _ in range(2)]
            hbuf = [torch.empty(nmax, dtype=torch.float64, pin_memory=True) for _ in range(2)]
            Dh = torch.empty(M, dtype=torch.float64, pin_memory=True)
            copy = torch.cuda.Stream(device=dev)
            done = [torch.cuda.Event() for _ in range(2)]
            ready = [torch.cuda.Event() for _ in range(2)]
            d2h = 0

            def e2e_step():
                nonlocal d2h
                d2h = M * 8
                h.update(cosmo, stream)
                h.spectra(D, stream)
                Dh.copy_(D, non_blocking=True)
                for k, (a, b) in enumerate(bands):
                    n = (packed_tiles(b) - packed_tiles(a)) * TILE * TILE
                    s = k % 2
                    stream.wait_event(done[s])
                    h.assemble_band(a, b - a, dbuf[s][:n], N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, prec, stream)
                    ready[s].record(stream)
                    copy.wait_event(ready[s])
                    with torch.cuda.stream(copy):
                        hbuf[s][:n].copy_(dbuf[s][:n], non_blocking=True)
                    done[s].record(copy)
                    d2h += n * 8
                copy.synchronize()
                stream.synchronize()

            e2e_step()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                e2e_step()
            e2e_s = (time.perf_counter() - t0) / args.steps
            del dbuf, hbuf
            # the FP64 GPU form on a sample of bands (the full FP64 contraction
            # at this size runs for many minutes): same rows, both precisions
            if not args.no_fp64_form and prec != N.COV_FP64:
                row0 = (M // 2) // TILE * TILE
                sample = [(row0, row0 + TILE), (M // TILE * TILE - TILE, M // TILE * TILE)]
                n = max(packed_tiles(b) - packed_tiles(a) for a, b in sample) * TILE * TILE
                buf = torch.empty(n, dtype=torch.float64, device=dev)
                res = {}
                for p, nm in ((prec, "split"), (N.COV_FP64, "fp64")):
                    def band_step(p=p):
                        for a, b in sample:
                            h.assemble_band(a, b - a, buf, N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, p, stream)
                    band_step()  # builds this precision's operands
                    ms_b, st_b, _ = timed(stream, band_step, 1, h, 1)
                    res[nm] = ms_b
                el = sum((b - a) * (a + b + 1) // 2 for a, b in sample)
                extra["fp64_form"] = {
                    "value": el / (res["fp64"] / 1e3), "unit": UNIT, "ms": res["fp64"],
                    "split_value_same_bands": el / (res["split"] / 1e3), "split_ms": res["split"],
                    "sample": f"rows {sample[0][0]}-{sample[0][1]} and {sample[1][0]}-{sample[1][1]} "
                              f"({el} lower elements, every term) in each precision"}
                del buf
        ms_step = ms_total / args.steps
        e2e = {"value": world * elements / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 56,
               "d2h_bytes_per_step": d2h,
               "how": f"cov_update + cov_spectra, then cov_assemble_band over {len(bands)} bands of about equal "
                      "size into two device buffers, each band copied to pinned host memory on a second stream "
                      "while the next one is assembled"}
        snr_sizes = []
        cfg = {"layout": "lower-packed 256x256 tiles, resident (%.1f GB)" % (Ct.numel() * 8 / 1e9)}
    else:
        with torch.cuda.stream(stream):
            clk.start()
            time.sleep(0.4)
            r = dense_run(h, wl, cosmo, prec, stream, args.steps, args.warmup, world, not args.no_fp64_form)
            clocks = clk.stop()
        ms_step, stages = r["ms_per_step"], r["stages"]
        D, C = r["D"], r["C"]
        which = (N.COV_WHICH_P, N.COV_WHICH_B, N.COV_WHICH_JOINT)
        Ch = torch.empty(M, M, dtype=torch.float64, pin_memory=True)
        Dh = torch.empty(M, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            for _ in range(args.steps):
                h.update(cosmo, stream)
                h.spectra(D, stream)
                h.assemble(C, N.COV_TERMS_ALL, prec, stream)
                [h.snr(C, D, w, stream) for w in which]
                Ch.copy_(C, non_blocking=True)
                Dh.copy_(D, non_blocking=True)
                stream.synchronize()
            e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = {"value": world * elements / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 56,
               "d2h_bytes_per_step": M * M * 8 + M * 8 + 3 * wl["bins"]["n_ell"] * 8}
        if "fp64" in r:
            extra["fp64_form"] = {"ms_per_step": r["fp64"]["ms_per_step"],
                                  "value": elements / (r["fp64"]["ms_per_step"] / 1e3), "unit": UNIT}
            extra["snr_rel_err_vs_fp64_form"] = r["snr_rel_err_vs_fp64_form"]
        extra["snr_joint_max"] = float(np.nanmax(r["snr"][2]))
        snr_sizes = [h.n_P, h.n_B, M]
        cfg = {"layout": "dense M x M"}

    ms_step = job_step_ms(ms_step, world, dev)
    value = world * elements / (ms_step / 1e3)
    roof = contraction_roofline(stages, elements, Kc, prec, N, long_kernel=packed, sm_mhz=clocks.get("sm_mhz"))
    if prec != N.COV_FP64:
        roof["traffic"] = measured_traffic(args.workload)
        roof["algorithmic_bytes"] = elements * 8 + 2 * 2 * M * Kc  # tiles written once, hi/lo operands read once
    if snr_sizes:
        chol_ms = stages["snr_cholesky"][0] / max(args.steps, 1)
        roof["cholesky"] = {"stage_ms_per_step": chol_ms,
                            "fp64_equivalent_tflops": sum(m ** 3 / 3.0 for m in snr_sizes) / (chol_ms / 1e3) / 1e12,
                            "note": "diagonal blocks and panel solves in FP64, trailing updates on tcgen05 by "
                                    "exact slicing"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == N.COV_FP64 else "bf16x3+f64",
           "data": "synthetic",
           "config": dict({"workload": args.workload, "M": M, "n_P": h.n_P, "n_B": h.n_B, "K": K,
                           "n_tomo": wl["nz"]["n_tomo"], "n_ell": wl["bins"]["n_ell"], "terms": "all",
                           "precision": prec_name, "elements_per_step": elements,
                           "step": "update+spectra+assemble" + ("" if packed else "+snr(P,B,joint)"),
                           "l2": "inputs larger than L2 (factor rows %.0f MB, covariance %.0f MB)" % (
                               M * Kc * (4 if prec != N.COV_FP64 else 8) / 1e6, elements * 8 / 1e6),
                           "parallelism": f"replicas x{world}"}, **cfg),
           "roofline": roof,
           "e2e": e2e,
           "gpu_launches": args.steps * launches_per_step(snr_sizes, h.n_tri, prec != N.COV_FP64, packed),
           "clocks": clocks,
           "stages_ms_per_step": {k: v[0] / max(args.steps, 1) for k, v in stages.items() if v[1]}}
    out.update(extra)
    h.close()
    if packed:
        del Ct
    torch.cuda.empty_cache()
    if not args.no_snr_run and packed and rank == 0:
        # the S/N stage (a dense FP64-accurate Cholesky per vector, P, B and
        # joint) on a workload whose dense square fits, timed in the same run,
        # with its error against the FP64 form and against the oracle's stored S/N
        wl2 = workloads.get(args.snr_workload)
        h2 = Handle(wl2, device=local, chol_kernel=chol)
        s2 = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s2):
            r2 = dense_run(h2, wl2, dict(wl2["cosmology"]), prec, s2, 3, 2, 1, True, fp64_steps=1)
        st = r2["stages"]
        M2 = h2.n_P + h2.n_B
        chol_ms = st["snr_cholesky"][0] / 3
        out["snr_stage"] = {
            "workload": args.snr_workload, "M": M2, "n_P": h2.n_P, "n_B": h2.n_B,
            "ms_per_full_step": r2["ms_per_step"],
            "full_step_elements_per_s": M2 * (M2 + 1) // 2 / (r2["ms_per_step"] / 1e3),
            "snr_ms_per_step": sum(st[k][0] for k in ("snr_pack", "snr_cholesky", "snr_prefix")) / 3,
            "cholesky_ms_per_step": chol_ms,
            "cholesky_fp64_equivalent_tflops": sum(m ** 3 / 3.0 for m in (h2.n_P, h2.n_B, M2)) / (chol_ms / 1e3) / 1e12,
            "snr_rel_err_vs_fp64_form": r2.get("snr_rel_err_vs_fp64_form"),
            "snr_joint_max": float(np.nanmax(r2["snr"][2]))}
        ref = stored_oracle_snr(args.snr_workload)
        if ref is not None:
            out["snr_stage"]["snr_rel_err_vs_oracle"] = {
                "split_bf16": max(max_rel(r2["snr"][k], ref[t]) for k, t in enumerate("PBJ")),
                "fp64_form": (max(max_rel(r2["fp64"]["snr"][k], ref[t]) for k, t in enumerate("PBJ"))
                              if "fp64" in r2 else None),
                "oracle": "tests/golden/snr_%s.txt (oracle FP64 covariance, scipy Cholesky)" % args.snr_workload}
        if "fp64" in r2:
            out["snr_stage"]["fp64_form_ms_per_full_step"] = r2["fp64"]["ms_per_step"]
        h2.close()
        del r2
        torch.cuda.empty_cache()
    if not args.no_snr_10bin and packed and rank == 0 and world == 1:
        # the joint S/N of the bench's own workload: a cumulative-order handle
        # assembles the packed tiles (plus the data row) and factorises them in place
        res = snr_tiles_run(workloads.get(args.workload), prec, local, [("joint", N.COV_ROWS_JOINT)], chol)
        j = res["joint"]
        out["snr_10bin"] = dict(j, precision=prec_name, workload=args.workload,
                                note="joint vector; P-only and B-only with --snr-10bin")
        torch.cuda.empty_cache()
    if not args.no_batch and packed and rank == 0 and world == 1:
        out["fisher_batch"] = batch_run(prec, local, [x for x in args.batch_bins.split(",") if x])
    if args.snr_10bin and rank == 0 and world == 1:
        sets = {"joint": N.COV_ROWS_JOINT, "B": N.COV_ROWS_B, "P": N.COV_ROWS_P}
        sp = prec if args.snr_precision == "auto" else (N.COV_FP64 if args.snr_precision == "fp64" else
                                                         N.COV_SPLIT_BF16)
        out["snr_tiles"] = snr_tiles_run(workloads.get(args.workload), sp, local,
                                         [(r, sets[r]) for r in args.snr_rows.split(",") if r], chol)
        out["snr_tiles"]["precision"] = "fp64" if sp == N.COV_FP64 else "split_bf16"
    if not args.no_pca and packed and rank == 0 and world == 1:
        try:
            out["pca"] = pca_run(local, [int(x) for x in args.pca_bins.split(",") if x])
        except Exception as e:  # noqa: BLE001
            out["pca"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_coupling and packed and rank == 0 and world == 1:
        try:
            out["coupling_exact"] = coupling_run(local, args.workload, "cfg2_5bin")
        except Exception as e:  # noqa: BLE001
            out["coupling_exact"] = {"error": f"{type(e).__name__}: {e}"}
    # optional stages: a failure is recorded in the line instead of losing it
    if args.model_a and rank == 0 and world == 1:
        try:
            out["model_a"] = model_a_run(prec, local, args.model_a_workload, args.model_a_nodes)
        except Exception as e:  # noqa: BLE001
            out["model_a"] = {"error": f"{type(e).__name__}: {e}"}
    if args.paper_replica and rank == 0 and world == 1:
        try:
            out["paper_replica"] = paper_run(local)
        except Exception as e:  # noqa: BLE001
            out["paper_replica"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_serve and packed and rank == 0 and world == 1:
        sv = serving_run(prec, args.serve_requests, args.serve_rate, args.serve_budget_gb, args.serve_slots, local)
        out["serving"] = {"workload": "Poisson stream (seed 2024), n_t uniform 1..10, n_ell uniform 8..24 on "
                                      "[10, 5000], cosmology within +-5% of the fiducial, N_chi=128, N_M=96, every "
                                      "term, covariance + 3 cumulative S/N per request",
                          "offered": sv}
        if args.serve_search:
            out["serving"]["search"] = serving_search(prec, args.serve_search_requests, args.serve_budget_gb,
                                                      args.serve_slots, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _has_split():
    try:
        from paper_1812_07437_gb300 import native
        return getattr(native, "HAS_SPLIT_BF16", False)
    except Exception:
        return False


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
