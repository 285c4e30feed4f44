"""Benchmark of the QMC hot path on GB300.

Headline (the `value`): materialised scrambled Sobol' points, s = 32
dimensions, 2^24 indices, hash-based nested scramble, u32 + fp32 outputs
(4 GiB written per step, larger than the 129 MB L2), in Gdims/s
(= 2^29 coordinates / step time).  One step = one qmc_sobol_points call.

Also reported in the same JSON line:
  e2e           the same metric through the C-ABI with host buffers: matrices
                and seeds copied in, both point arrays copied back to pinned
                host memory, every step
  roofline      the point kernel against the measured HBM copy bandwidth
  cpu_baseline  the oracle on a bounded sample, on the host's cores
  fused         fused forward+backward of the differentiable integro-
                approximation (1024x1024 integrals x 4096 samples), the
                unfused forward + backward kernels, the batched 1920x1080
                integration and the fused rank-1 lattice Genz integration,
                each in Gsamples/s with its error against the oracle on a
                sample of results

--impl reference times the oracle (the plain CPU reference of the same
computation) on a bounded sample of the headline workload.
Under torchrun every rank materialises its own index window (weak scaling,
no collective on the data path); rank 0 prints the line.
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

METRIC = "scrambled Sobol Gdims/s; fused QMC fwd+bwd Gsamples/s at stated err, % roofline"
S_DIMS, N_POINTS = 32, 1 << 24


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="headline only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--log2-points", type=int, default=24, help="points per GPU (2^k); 24 is the workload")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_window(rank: int, world: int, n: int = N_POINTS):
    """Index window of one rank: rank r materialises indices [r n, (r+1) n)."""
    return rank * n, n


# ------------------------------------------------------------------ peaks, clocks
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = {"sobol_points_fast<1,2>": ["points.cu", "qmc_device.cuh", "qmc_internal.h"]}


def profile_traffic(kernel_key: str):
    """dram bytes per launch from the committed ncu summary, or None when the
    kernel's sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    from paper_2307_15584_gb300.build import source_digest

    digest = source_digest(KERNEL_SOURCES[kernel_key])
    for line in open(path):
        parts = line.split()
        if len(parts) == 3 and parts[0] == kernel_key and parts[1] == digest:
            return float(parts[2])
    return None


# ------------------------------------------------------------------ oracle baseline
def cpu_baseline(n_rows: int = 1 << 23):
    import oracle
    from paper_2307_15584_gb300 import inputs

    C = oracle.sobol_matrices(S_DIMS, inputs.sobol_raw_init(S_DIMS))
    seeds = inputs.scramble_seeds(S_DIMS)
    threads = os.cpu_count() or 1
    oracle.sobol_points(C, 0, 1024, oracle.SCRAMBLE_NESTED, seeds, threads=threads)
    t0 = time.perf_counter()
    oracle.sobol_points(C, 0, n_rows, oracle.SCRAMBLE_NESTED, seeds, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n_rows * S_DIMS / dt / 1e9, "unit": "Gdims/s", "cores": threads, "kind": "oracle",
            "sample": f"{n_rows} points x {S_DIMS} dims (nested scramble, u32+fp32) of the 2^24-point workload",
            "seconds": dt}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    from paper_2307_15584_gb300 import inputs

    C = oracle.sobol_matrices(S_DIMS, inputs.sobol_raw_init(S_DIMS))
    seeds = inputs.scramble_seeds(S_DIMS)
    threads = os.cpu_count() or 1
    rows = 1 << 14
    for _ in range(args.warmup):
        oracle.sobol_points(C, 0, rows, oracle.SCRAMBLE_NESTED, seeds, threads=threads)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.sobol_points(C, k * rows, rows, oracle.SCRAMBLE_NESTED, seeds, threads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = rows * S_DIMS / (ms * 1e-3) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gdims/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"scrambled Sobol s={S_DIMS}, sample of {rows} points per step "
                                   f"(full workload 2^24 points), nested scramble, u32+fp32", "s": S_DIMS,
                       "points_per_step": rows},
            "cpu_baseline": {"value": value, "unit": "Gdims/s", "cores": threads, "kind": "oracle",
                             "sample": f"{rows} points x {S_DIMS} dims per step"},
            "e2e": {"value": value, "unit": "Gdims/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arms
def timed(fn, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    start = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    end = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        start[k].record(stream)
        fn()
        end[k].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(start, end)]


def bench_extra(dev, steps, warmup):
    """Integration workloads: throughput and error against the oracle on a sample."""
    import torch

    import oracle
    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    stream = torch.cuda.current_stream()
    out = {}
    rng = np.random.default_rng(1)

    # -- differentiable integro-approximation: 1024x1024 x 4096, fused fwd+bwd
    n = 1 << 20
    counts = np.full(n, 4096, np.uint32)
    C6 = B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6))
    theta = inputs.gaussmix_theta(n)
    seeds = inputs.pixel_seeds(n, 6)
    target = inputs.gaussmix_target(inputs.gaussmix_theta(n, seed=inputs.DEFAULT_SEED + 1))
    d = {"C": B.u32_tensor(C6, dev), "c": B.u32_tensor(counts, dev), "th": torch.from_numpy(theta).to(dev),
         "sd": B.u32_tensor(seeds, dev), "tg": torch.from_numpy(target).to(dev)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"], seeds=d["sd"],
                          seeds_per_integral=True, with_gradient=True)
    ws = B.alloc_workspace(prob, n, counts, dev)
    est = torch.empty(n, dtype=torch.float64, device=dev)
    gth = torch.empty((n, 16), dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    ge = torch.empty(n, dtype=torch.float64, device=dev)
    gb = torch.empty((n, 16), dtype=torch.float32, device=dev)

    def fused():
        B.qmc_integrate_fwd_bwd(prob, n, d["c"], d["th"], d["tg"], est, gth, loss, ws)

    def unfused():
        B.qmc_integrate(prob, n, d["c"], d["th"], est, ws)
        torch.sub(est, d["tg"], out=ge).mul_(2.0)
        B.qmc_integrate_backward(prob, n, d["c"], d["th"], ge, gb, ws)

    samples = float(counts.sum())
    tf = timed(fused, steps, warmup, stream)
    tu = timed(unfused, max(2, steps // 2), 2, stream)
    fused()
    torch.cuda.synchronize()
    pix = np.sort(rng.choice(n, 64, replace=False))
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts[pix], theta[pix], C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds[pix], with_grad=True)
    e = est.cpu().numpy()[pix]
    g = gth.cpu().numpy()[pix]
    r = ref["est"] - target[pix]
    g_ref = 2 * r[:, None] * ref["grad"]
    g_scale = 2 * np.abs(r)[:, None] * (np.abs(ref["grad"]) + ref["grad_mass"])
    out["fwd_bwd_1024x1024x4096"] = {
        "fused_gsamples_s": samples / (statistics.median(tf) * 1e-3) / 1e9,
        "unfused_gsamples_s": samples / (statistics.median(tu) * 1e-3) / 1e9,
        "fused_ms": statistics.median(tf), "unfused_ms": statistics.median(tu),
        "est_max_rel_err_vs_oracle": float(np.max(np.abs(e - ref["est"]) / np.abs(ref["est"]))),
        "grad_max_err_over_scale": float(np.max(np.abs(g - g_ref) / np.maximum(g_scale, 1e-300))),
        "oracle_sample_pixels": int(pix.size)}
    del ws, est, gth, gb, d
    torch.cuda.empty_cache()

    # -- batched 1920x1080, log-uniform counts in [1, 65536]
    n = 1920 * 1080
    counts = inputs.log_uniform_counts(n)
    theta = inputs.gaussmix_theta(n, seed=7)
    seeds = inputs.pixel_seeds(n, 6, seed=7)
    d = {"C": B.u32_tensor(C6, dev), "c": B.u32_tensor(counts, dev), "th": torch.from_numpy(theta).to(dev),
         "sd": B.u32_tensor(seeds, dev)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"], seeds=d["sd"],
                          seeds_per_integral=True)
    ws = B.alloc_workspace(prob, n, counts, dev)
    est = torch.empty(n, dtype=torch.float64, device=dev)

    def batched():
        B.qmc_integrate(prob, n, d["c"], d["th"], est, ws)

    tb = timed(batched, max(2, steps // 2), 2, stream)
    batched()
    torch.cuda.synchronize()
    pix = np.sort(rng.choice(n, 256, replace=False))
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts[pix], theta[pix], C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds[pix])
    e = est.cpu().numpy()[pix]
    W = np.abs(theta[pix][:, 0::4]).sum(axis=1)
    err = np.abs(e - ref["est"])
    out["batched_1920x1080"] = {
        "gsamples_s": float(counts.sum()) / (statistics.median(tb) * 1e-3) / 1e9, "ms": statistics.median(tb),
        "samples": int(counts.sum()),
        "max_rel_err_vs_oracle": float(np.max(err / np.maximum(np.abs(ref["est"]), 1e-300))),
        "within_tol": int((err <= 1e-6 * np.abs(ref["est"]) + 1e-12 * W).sum()), "oracle_sample_pixels": int(pix.size)}
    del ws, est, d
    torch.cuda.empty_cache()

    # -- rank-1 lattice s = 16, 2^26 points, Genz product peak + oscillatory, 4 sets each
    s, N = 16, 1 << 26
    g, sh = inputs.lattice_generator(s), inputs.lattice_shift(s)
    res = {}
    for fam, kind in (("product_peak", B.F_GENZ_PRODUCT_PEAK), ("oscillatory", B.F_GENZ_OSCILLATORY)):
        theta = np.stack([inputs.genz_params(fam, s, k) for k in range(4)])
        counts = np.full(4, N, np.uint32)
        d = {"g": B.u32_tensor(g, dev), "sh": B.u32_tensor(sh, dev), "c": B.u32_tensor(counts, dev),
             "th": torch.from_numpy(theta).to(dev)}
        prob = B.make_problem(B.SOURCE_LATTICE, kind, s, 0, g=d["g"], seeds=d["sh"])
        ws = B.alloc_workspace(prob, 4, counts, dev)
        est = torch.empty(4, dtype=torch.float64, device=dev)
        tl = timed(lambda: B.qmc_integrate(prob, 4, d["c"], d["th"], est, ws), max(2, steps // 2), 2, stream)
        e = est.cpu().numpy()
        exact = np.array([oracle.exact_genz_product_peak(t, s) if fam == "product_peak"
                          else oracle.exact_genz_oscillatory(t, s) for t in theta])
        res[fam] = {"gsamples_s": 4.0 * N / (statistics.median(tl) * 1e-3) / 1e9, "ms": statistics.median(tl),
                    "rel_err_vs_exact": [float(v) for v in np.abs(e - exact) / np.abs(exact)]}
    out["lattice_genz_s16_2p26"] = res
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()

    begin, count = rank_window(rank, world, 1 << args.log2_points)
    C = B.qmc_sobol_matrices(S_DIMS, inputs.sobol_raw_init(S_DIMS))
    seeds = inputs.scramble_seeds(S_DIMS)
    Cd, sd = B.u32_tensor(C, dev), B.u32_tensor(seeds, dev)
    out_u = torch.empty((count, S_DIMS), dtype=torch.int32, device=dev)
    out_f = torch.empty((count, S_DIMS), dtype=torch.float32, device=dev)

    def step():
        B.qmc_sobol_points(Cd, S_DIMS, begin, count, B.SCRAMBLE_NESTED, sd, out_u, out_f)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    per = []
    for k in range(args.steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms = total_ms / args.steps
    coords = float(count) * S_DIMS * world
    value = coords / (ms * 1e-3) / 1e9

    # end to end through the C-ABI from host buffers
    h_C = torch.from_numpy(C.view(np.int32)).pin_memory()
    h_s = torch.from_numpy(seeds.view(np.int32)).pin_memory()
    h_u = torch.empty((count, S_DIMS), dtype=torch.int32).pin_memory()
    h_f = torch.empty((count, S_DIMS), dtype=torch.float32).pin_memory()

    def e2e_step():
        Cd.copy_(h_C, non_blocking=True)
        sd.copy_(h_s, non_blocking=True)
        step()
        h_u.copy_(out_u, non_blocking=True)
        h_f.copy_(out_f, non_blocking=True)

    te = timed(e2e_step, 3, 1, stream)
    e2e_ms = statistics.median(te)
    h2d = h_C.numel() * 4 + h_s.numel() * 4
    d2h = h_u.numel() * 4 + h_f.numel() * 4

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    kernel_ms = statistics.mean(per)
    bytes_per_launch = float(count) * S_DIMS * 8
    achieved = bytes_per_launch / (kernel_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Gdims/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "materialised scrambled Sobol: s=32 dims, 2^24 indices per GPU, nested scramble, "
                               "u32+fp32 outputs [2^24][32] each", "s": S_DIMS, "points_per_gpu": count,
                   "scramble": "nested", "outputs": "u32+f32",
                   "l2": "outputs (4 GiB per step) exceed the 129 MB L2; no flush needed"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": profile_traffic("sobol_points_fast<1,2>"),
                     "peak_source": peaks["source"] + " copy bandwidth",
                     "algorithmic_bytes_per_launch": bytes_per_launch},
        "e2e": {"value": coords / (e2e_ms * 1e-3) / 1e9, "unit": "Gdims/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    del out_u, out_f, h_u, h_f
    torch.cuda.empty_cache()
    if not args.no_extra:
        line["fused"] = bench_extra(dev, 5, 3)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
