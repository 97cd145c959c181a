#!/usr/bin/env python
"""Benchmark of the joint P+B covariance path on GB300.

One step = the whole path for one cosmology of the workload: device tables
and exact counts (cov_update), spectra and data vector (cov_spectra), the full
joint covariance with every term (cov_assemble) and the cumulative S/N of P,
B and the joint vector (three cov_snr calls, FP64 Cholesky).  The metric is
unique covariance elements M(M+1)/2 per second.

Default workload: cfg2_5bin (5 tomographic bins, 12 ell bins on [10, 5000],
N_chi = 128, N_M = 96, M = 6375).  With --gpus N > 1 (torchrun) each rank runs
its own cosmology of a Fisher-style set (weak scaling, no collective on the
data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|split_bf16]
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
    p.add_argument("--workload", default="cfg2_5bin")
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "split_bf16"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-form", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    return p.parse_args()


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


def cpu_baseline(name, seconds):
    r, t_build = oracle_run(name)
    a, b = oracle_elements(r, 200000, 1234)
    t0 = time.perf_counter()
    n = 0
    while n < len(a) and time.perf_counter() - t0 < seconds:
        r.cov.element(int(a[n]), int(b[n]))
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} seeded lower-triangle elements of {name} (M={r.M}), every term, per-element "
                      f"oracle sums in {dt:.1f} s on 1 host core; oracle tables/spectra build "
                      f"{t_build:.1f} s not included"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    r, t_build = oracle_run(args.workload)
    per_step = 400
    a, b = oracle_elements(r, per_step * (args.steps + args.warmup), 4321)
    k = 0
    for _ in range(args.warmup):
        for _ in range(per_step):
            r.cov.element(int(a[k]), int(b[k]))
            k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(per_step):
            r.cov.element(int(a[k]), int(b[k]))
            k += 1
    dt = time.perf_counter() - t0
    v = per_step * args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "M": r.M, "sample_per_step": per_step},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{per_step} seeded covariance elements per step of {args.workload}; "
                                      f"oracle build {t_build:.1f} s not timed"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


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
def launches_per_step(which_sizes, n_tri, split):
    """Kernels of libwlcov launched by one step (memsets not counted)."""
    tables = 11          # chi_max, los, growth_norm, amplitude, sigma, halo, profiles, edges, norms, kernels, sigw2
    counts = 3 if n_tri > 0 else 2
    spectra = 5 if n_tri > 0 else 3
    assemble = 7         # split: rows_t, split(T), tc(T), rows_prep, rows_split, tc(1h+SSC), gather
    snr = 0              # FP64: rows_t, gemm(T), rows_a, gemm(1h), gather, rows_s, gemm(SSC)
    for ms in which_sizes:
        nb = (ms + 63) // 64
        snr += 2 + 4 * nb  # pack, prefix; per panel: diagonal block, panel solve, slice, tensor-core update
    return tables + counts + spectra + assemble + snr


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

    wl = workloads.get(args.workload)
    cosmo = dict(wl["cosmology"])
    if rank > 0:  # Fisher-style +-1% steps, one cosmology per rank
        keys = ["Om", "sigma8", "h", "ns", "Ob", "w0"]
        k = keys[(rank - 1) % len(keys)]
        cosmo[k] *= 1.0 + 0.01 * (1 if rank % 2 else -1)
        wl = workloads.get(args.workload, cosmology=cosmo)
    h = Handle(wl, device=local)
    M = h.M
    elements = M * (M + 1) // 2
    D = torch.zeros(M, dtype=torch.float64, device=dev)
    C = torch.zeros(M, M, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    which = (N.COV_WHICH_P, N.COV_WHICH_B, N.COV_WHICH_JOINT)

    def step():
        h.update(cosmo, stream)
        h.spectra(D, stream)
        h.assemble(C, N.COV_TERMS_ALL, prec, stream)
        return [h.snr(C, D, w, stream) for w in which]

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            snr = step()
        torch.cuda.synchronize()
        h.profile(True)
        h.stage_times()
        gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or 0) \
            if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
        clk = ClockSampler(gpu_index)
        clk.start()
        time.sleep(0.4)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            snr = step()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms_total = e0.elapsed_time(e1)
        clocks = clk.stop()
        stages = h.stage_times()
        h.profile(False)

        # end-to-end through the public API with host buffers: parameters in,
        # covariance + data vector + S/N out to pinned host memory every step
        Ch = torch.empty(M, M, dtype=torch.float64, pin_memory=True)
        Dh = torch.empty(M, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
            Ch.copy_(C, non_blocking=True)
            Dh.copy_(D, non_blocking=True)
            stream.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps

        # the plain FP64 form of the same step (the comparison point of the
        # reduced-precision form): a short timed run after the main one
        fp64 = None
        if prec != N.COV_FP64 and not args.no_fp64_form:
            def step64():
                h.update(cosmo, stream)
                h.spectra(D, stream)
                h.assemble(C, N.COV_TERMS_ALL, N.COV_FP64, stream)
                return [h.snr(C, D, w, stream) for w in which]
            step64()
            torch.cuda.synchronize()
            h.profile(True)
            h.stage_times()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(2):
                step64()
            f1.record(stream)
            torch.cuda.synchronize()
            st64 = h.stage_times()
            h.profile(False)
            ms64 = f0.elapsed_time(f1) / 2
            s1h = st64["syrk_1h"][0] / max(st64["syrk_1h"][1], 1)
            fp64 = {"ms_per_step": ms64, "value": elements / (ms64 / 1e3), "unit": UNIT,
                    "syrk_1h_ms": s1h, "syrk_1h_tflops": 2.0 * elements * wl["bins"]["n_chi"]
                    * wl["bins"]["n_mass"] / (s1h / 1e3) / 1e12}

    t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_step = float(t.item()) / args.steps
    value = world * elements / (ms_step / 1e3)

    # roofline of the 1-halo (chi, M) contraction, the kernel the metric is built on
    syrk_ms, syrk_calls = stages["syrk_1h"]
    K = wl["bins"]["n_chi"] * wl["bins"]["n_mass"]
    if prec != N.COV_FP64:
        K += wl["bins"]["n_chi"]  # the super-sample rows ride along in the split contraction
    flops = 2.0 * elements * K
    avg_ms = syrk_ms / max(syrk_calls, 1)
    achieved = flops / (avg_ms / 1e3) / 1e12
    if prec == N.COV_FP64:
        roof = {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                "frac": achieved / 1.25, "traffic": None, "kernel": "k_gemm_lower (FP64 1-halo contraction)",
                "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak available)"}
    else:
        import json as _j
        peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak = peaks["bf16_tflops"]
        issued = 3.0 * flops
        roof = {"bound": "tensor", "achieved": issued / (avg_ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": issued / (avg_ms / 1e3) / 1e12 / peak, "traffic": None,
                "kernel": "k_syrk_tc (tcgen05 split-BF16 1-halo contraction)",
                "algorithmic_tflops": achieved, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"}

    sizes = [h.n_P, h.n_B, M]
    # the S/N factorisations hold most of the step: report their tensor-core
    # trailing update too (FP64-equivalent work M^3/3 per factorisation)
    chol_ms = stages["snr_cholesky"][0] / max(args.steps, 1)
    chol_flops = sum(m ** 3 / 3.0 for m in sizes)
    roof["cholesky"] = {"stage_ms_per_step": chol_ms, "fp64_equivalent_tflops": chol_flops / (chol_ms / 1e3) / 1e12,
                        "note": "diagonal blocks and panel solves in FP64, trailing updates on tcgen05 by exact slicing"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == N.COV_FP64 else "bf16x3+f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "M": M, "n_P": h.n_P, "n_B": h.n_B, "K": K,
                      "n_tomo": wl["nz"]["n_tomo"], "n_ell": wl["bins"]["n_ell"], "terms": "all",
                      "precision": prec_name, "elements_per_step": elements,
                      "l2": "inputs larger than L2 (factor rows %.0f MB, covariance %.0f MB)" % (
                          M * K * 8 / 1e6, M * M * 8 / 1e6),
                      "parallelism": f"replicas x{world}"},
           "roofline": roof,
           "e2e": {"value": world * elements / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 56,
                   "d2h_bytes_per_step": M * M * 8 + M * 8 + 3 * wl["bins"]["n_ell"] * 8},
           "gpu_launches": args.steps * launches_per_step(sizes, h.n_tri, prec != N.COV_FP64),
           "fp64_form": fp64,
           "clocks": clocks,
           "stages_ms_per_step": {k: v[0] / max(args.steps, 1) for k, v in stages.items()},
           "snr_joint_max": float(np.nanmax(snr[2]))}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    h.close()
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
