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
  cpu_baseline  the oracle on a bounded sample, on the host's cores (and, inside
                each extra below, the oracle on a bounded sample of that
                workload)
  fused         (last, a summary; --detail-out FILE writes every figure) the fused
                forward+backward of the differentiable integro-approximation
                (1024x1024 integrals x 4096 samples) against the unfused forward
                + backward kernels, with its estimates' and gradients' errors
                against the oracle on 1024 of the pixels; the batched 1920x1080
                integration; the rank-1 lattice Genz integration (fused, and
                unfused through 4 GiB of materialised points); one integral of
                16 (2^32 - 1) samples over the elements of a partitioned 64-bit
                Sobol' sequence -- each in Gsamples/s with its issue roofline
                (alg_frac: the method's operations per sample; issue_frac: the
                executed instructions; pipes: per-pipe ncu figures) and the
                oracle's rate on all host cores and on one core; and every
                materialising point generator on the headline shape (Gdims/s,
                fraction of the measured copy bandwidth)

--only {fwd_bwd,batched,lattice,points,partition,samplers} --small runs one extra workload alone at
a reduced size (for ncu captures; samplers -- the Fig. 1 substitute -- runs only this way);
--impl reference times the oracle (the plain CPU reference of the same computation) on a
bounded sample of the headline workload.  Under torchrun every rank materialises its own index window (weak
scaling, no collective on the data path), or with --plan partition its own
element of the sequence partitioned by an extra dimension; rank 0 prints the
line.  The oracle runs only in the cpu_baseline and reference legs.
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
SMS, SCHEDULERS_PER_SM, WARP = 152, 4, 32  # GB300: one warp-instruction per scheduler per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="headline only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--log2-points", type=int, default=24, help="points per GPU (2^k); 24 is the workload")
    ap.add_argument("--only", choices=["fwd_bwd", "batched", "lattice", "points", "samplers", "partition"],
                    default=None,
                    help="run one extra workload alone (no headline)")
    ap.add_argument("--small", action="store_true", help="reduced integration sizes (profiling)")
    ap.add_argument("--detail-out", default=None,
                    help="write every figure of the extra workloads (the JSON line keeps a summary) to this file")
    ap.add_argument("--plan", choices=["window", "partition"], default="window",
                    help="per-rank work: a contiguous index window, or one element of the sequence "
                         "partitioned by its phi_2 dimension across the ranks (Sec. 2.5.1)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_window(rank: int, world: int, n: int = N_POINTS):
    """Index window of one rank: rank r materialises indices [r n, (r+1) n)."""
    return rank * n, n


def rank_partition(rank: int, world: int):
    """Element of the partitioned sequence that a rank enumerates (Sec. 2.5.1):
    (q, p) with P = 2^q = world and p = rank; element p owns the indices
    J 2^q + (q-bit reversal of p)."""
    if world < 1 or world & (world - 1) or not 0 <= rank < world:
        raise ValueError("the partition plan needs a power-of-two number of ranks")
    return world.bit_length() - 1, rank


# ------------------------------------------------------------------ peaks, clocks, profiles
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


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


POINTS_SOURCES = ["sobol_points.cu", "points_common.cuh", "qmc_device.cuh", "qmc_internal.h"]
INTEGRATE_COMMON = ["integrate_kernel.cuh", "qmc_device.cuh", "qmc_integrate.h", "qmc_internal.h"]


def integrate_sources(key: str) -> list[str]:
    """Sources of the fused kernel a profile figure belongs to: its integrand's
    translation unit and the shared kernel header."""
    unit = "integrate_gaussmix.cu" if "gaussmix" in key else "integrate_genz.cu"
    return [unit] + INTEGRATE_COMMON
KERNEL_SOURCES = {"sobol_points_fast<1,2>": POINTS_SOURCES}
POINTS_COMMON = ["points_common.cuh", "qmc_device.cuh", "qmc_internal.h"]
# the points workloads' kernels: (profile key, the kernel's own sources besides POINTS_COMMON)
POINTS_KERNELS = {"sobol32_nested": ("sobol_points_fast<1,2>", ["sobol_points.cu"]),
                  "sobol32_nested_from_index_1": ("sobol_points_fast<1,2>@1", ["sobol_points.cu"]),
                  "sobol40_nested": ("sobol_points_walk<2>", ["sobol_points.cu"]),
                  "lattice_shifted": ("lattice_points_fast<1,0,1>", ["lattice_points.cu"]),
                  "lattice_shifted_from_index_1": ("lattice_points_flat<0>", ["lattice_points.cu"]),
                  "halton_faure": ("halton_points_kernel<faure>", ["halton_points.cu", "halton_points.h"]),
                  "pixel_lattice_16spp": ("pixel_lattice_points_fast", ["lattice_points.cu"]),
                  "random_lattice_hash_x4_16spp": ("random_lattice_points_fast<hash>", ["lattice_points.cu"]),
                  "random_lattice_lfsr_x4_16spp": ("random_lattice_points_fast<lfsr>", ["lattice_points.cu"])}


def profile_sources(fname: str, key: str) -> list[str]:
    """The sources whose digest keys a committed profile figure."""
    if fname == "traffic.txt":
        return KERNEL_SOURCES[key]
    if fname in ("inst_per_sample.txt", "pipes.txt"):
        return integrate_sources(key)
    for k, src in POINTS_KERNELS.values():
        if k == key:
            return src + POINTS_COMMON
    raise KeyError(key)


def _profile_value(fname: str, key: str, files):
    """A per-kernel figure from a committed profile summary, or None when the
    kernel's sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None
    from paper_2307_15584_gb300.build import source_digest

    digest = source_digest(files)
    for line in open(path):
        parts = line.split()
        if len(parts) == 3 and parts[0] == key and parts[1] == digest:
            return float(parts[2])
    return None


def profile_traffic(kernel_key: str):
    return _profile_value("traffic.txt", kernel_key, KERNEL_SOURCES[kernel_key])


# Operations per sample that the method itself needs in each fused workload (not what the
# kernel executes): per coordinate of a nested-scrambled Sobol' point about 15 integer
# operations (the column XOR, the hash steps, the float conversion); the 6-D mixture
# 4 x (6 FSUB + 6 FFMA) + 4 ex2 and a 4-operation compensated add (146 per sample), its
# gradient 4 x (6 + 3) more FMAs (182); per lattice coordinate one IMAD, one IADD, one
# conversion with one brev per point; the product peak 16 x (FADD + FFMA + FMUL) and one
# reciprocal (98 per sample in all), the oscillatory 16 FFMAs and one cosine (66).  The
# partitioned 64-bit workload has no such count (its alg_frac is null; its issue fraction
# stands alone).
ALG_OPS_PER_SAMPLE = {"integrate_main<sobol6,nested,gaussmix,grad>": 182.0,
                      "integrate_main<sobol6,nested,gaussmix>": 146.0,
                      "integrate_main<lattice16,product_peak>": 98.0,
                      "integrate_main<lattice16,oscillatory>": 66.0}
PIPES = ("alu", "fma", "fmaheavy", "xu")


def _profile_row(fname: str, key: str, files):
    """All numeric fields after the digest of a digest-keyed profile line, or None."""
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None
    from paper_2307_15584_gb300.build import source_digest

    digest = source_digest(files)
    for line in open(path):
        parts = line.split("#", 1)[0].split()  # a trailing comment is not a figure
        if len(parts) >= 3 and parts[0] == key and parts[1] == digest:
            return [float(v) for v in parts[2:]]
    return None


def issue_roofline(samples_per_s: float, key: str, sm_mhz):
    """Instruction-issue roofline of a fused integration kernel against SMs x schedulers x
    32 lanes x SM clock, two ways: `alg_frac` counts the method's own operations per sample
    (ALG_OPS_PER_SAMPLE), `frac` the thread-instructions the kernel executes per sample
    (ncu, profiles/inst_per_sample.txt); `pipes` = the fraction of each pipe's peak the
    kernel kept busy (ncu, profiles/pipes.txt)."""
    ips = _profile_value("inst_per_sample.txt", key, integrate_sources(key))
    clock = sm_mhz or measured_peaks()["sm_max_mhz"]
    peak = SMS * SCHEDULERS_PER_SM * WARP * clock * 1e6 / 1e9  # Ginst/s
    alg = ALG_OPS_PER_SAMPLE.get(key)
    out = {"bound": "alu", "peak": peak, "unit": "Ginst/s", "kernel": key, "clock_mhz": clock,
           "alg_ops_per_sample": alg, "alg_achieved": None if alg is None else samples_per_s * alg / 1e9,
           "alg_frac": None if alg is None else samples_per_s * alg / 1e9 / peak, "inst_per_sample": ips,
           "achieved": None if ips is None else samples_per_s * ips / 1e9,
           "frac": None if ips is None else samples_per_s * ips / 1e9 / peak}
    pipes = _profile_row("pipes.txt", key, integrate_sources(key))
    out["pipes"] = None if pipes is None else dict(zip(PIPES, pipes))
    return out


# ------------------------------------------------------------------ oracle baseline
def _discard(_result) -> None:
    """Drops a sample's outputs (the rate is what is wanted)."""
    return None


def _oracle_rates(run, units: float, unit: str, sample: str, one_core_fraction: int = 16) -> dict:
    """The oracle as it stands on a bounded sample: run(k, threads) computes the sample's
    first 1/k of the units on `threads` host threads.  Timed once on every host core
    (`value`, `cores`) and once on a single core over 1/one_core_fraction of the units
    (`value_1core`)."""
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    res = run(1, threads)
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    run(one_core_fraction, 1)
    d1 = time.perf_counter() - t1
    out = {"value": units / dt / 1e9, "unit": unit, "cores": threads, "kind": "oracle", "sample": sample,
           "seconds": dt, "value_1core": units / one_core_fraction / d1 / 1e9,
           "sample_1core": f"the first 1/{one_core_fraction} of it on one core", "seconds_1core": d1}
    return out if res is None else {**out, "_result": res}


def cpu_baseline(n_rows: int = 1 << 23):
    import oracle
    from paper_2307_15584_gb300 import inputs

    C = oracle.sobol_matrices(S_DIMS, inputs.sobol_raw_init(S_DIMS))
    seeds = inputs.scramble_seeds(S_DIMS)
    oracle.sobol_points(C, 0, 1024, oracle.SCRAMBLE_NESTED, seeds)
    def run(k, t):
        return _discard(oracle.sobol_points(C, 0, n_rows // k, oracle.SCRAMBLE_NESTED, seeds, threads=t))

    return _oracle_rates(run, n_rows * S_DIMS, "Gdims/s",
                         f"{n_rows} points x {S_DIMS} dims (nested scramble, u32+fp32) of the 2^24-point workload")


def extras_cpu_baselines(names) -> dict:
    """The oracle as it stands on a bounded sample of each extra workload (the same
    inputs, seeds and shapes; a fraction of the units), on all host cores and on one
    core: the CPU figures beside each GPU figure.  About 20 s in all on 16 cores.  The
    fused forward+backward sample keeps the oracle's results, to state the GPU's
    errors against them."""
    import oracle
    from paper_2307_15584_gb300 import inputs

    out = {}
    if "fwd_bwd" in names:  # config 5: 1024 of the 2^20 pixels x 4096 samples, estimate and gradient
        n = 1024
        C6 = oracle.sobol_matrices(6, inputs.sobol_raw_init(6))
        th, sd = inputs.gaussmix_theta(1 << 20)[:n], inputs.pixel_seeds(n, 6)
        out["fwd_bwd"] = _oracle_rates(
            lambda k, t: oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6,
                                          np.full(n // k, 4096, np.uint32), th[:n // k], C=C6,
                                          scramble=oracle.SCRAMBLE_NESTED, seeds=sd[:n // k], with_grad=True,
                                          threads=t),
            n * 4096.0, "Gsamples/s", f"{n} of the 2^20 pixels x 4096 samples, estimate + gradient")
    if "batched" in names:  # config 4: the first 1024 of the 1920x1080 pixels, their log-uniform counts
        n = 1024
        counts = inputs.log_uniform_counts(1920 * 1080)[:n]
        C6 = oracle.sobol_matrices(6, inputs.sobol_raw_init(6))
        th, sd = inputs.gaussmix_theta(1920 * 1080, seed=7)[:n], inputs.pixel_seeds(n, 6, seed=7)
        k1 = 16
        def batched(k, t):
            return _discard(oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts[:n // k],
                                             th[:n // k], C=C6, scramble=oracle.SCRAMBLE_NESTED, seeds=sd[:n // k],
                                             threads=t))

        out["batched"] = _oracle_rates(batched, float(counts.sum()), "Gsamples/s",
                                       f"the first {n} of the 1920x1080 pixels ({int(counts.sum())} samples)",
                                       one_core_fraction=k1)
        # the single-core sample's own sample count: the first n / k1 pixels' counts
        out["batched"]["value_1core"] *= float(counts[:n // k1].sum()) / (float(counts.sum()) / k1)
    if "lattice" in names:  # config 3: 4 integrals x 2^20 of the 2^26 points, per family
        s, N = 16, 1 << 20
        g, sh = inputs.lattice_generator(s), inputs.lattice_shift(s)
        res = {}
        for fam, kind in (("product_peak", oracle.F_GENZ_PRODUCT_PEAK), ("oscillatory", oracle.F_GENZ_OSCILLATORY)):
            th = np.stack([inputs.genz_params(fam, s, k) for k in range(4)])
            def lattice(k, t, th=th, kind=kind):
                return _discard(oracle.integrate(oracle.SOURCE_LATTICE, kind, s, np.full(4, N // k, np.uint32), th,
                                                 g=g, seeds=sh, threads=t))

            res[fam] = _oracle_rates(lattice, 4.0 * N, "Gsamples/s", "4 integrals x 2^20 of the 2^26 points")
        out["lattice"] = res
    if "partition" in names:  # the 16 elements x 2^16 of their 2^32 - 1 samples
        s, q, n = 16, 4, 1 << 16
        W = oracle.sobol_matrices_wide(s + 1, 64, inputs.sobol_raw_init(s + 1))
        th = inputs.genz_params("product_peak", s, 0)
        def partition(k, t):
            return _discard(oracle.integrate_partitioned(oracle.F_GENZ_PRODUCT_PEAK, s, np.full(16, n // k, np.uint32),
                                                         np.tile(th, (16, 1)), W, q, np.arange(16),
                                                         scramble=oracle.SCRAMBLE_NESTED,
                                                         seeds=inputs.scramble_seeds(s), threads=t))

        out["partition"] = _oracle_rates(partition, 16.0 * n, "Gsamples/s",
                                         "the 16 elements x 2^16 of their 2^32 - 1 samples")
    if "points" in names:  # every generator on s = 32, 2^10 .. 2^20 rows (about half a second each)
        s, n, nl = S_DIMS, 1 << 18, 1 << 10
        nb = 1 << 20
        C = oracle.sobol_matrices(s, inputs.sobol_raw_init(s))
        W = oracle.sobol_matrices_wide(s + 1, 64, inputs.sobol_raw_init(s + 1))
        sd = inputs.scramble_seeds(s)
        C37 = oracle.sobol_matrices(37, inputs.sobol_raw_init(37))
        C40, sd40 = np.concatenate([C37, C37[:3]]), inputs.scramble_seeds(40)
        g, sh = inputs.lattice_generator(s), inputs.lattice_shift(s)
        nested = oracle.SCRAMBLE_NESTED
        runs = {
            "sobol32_nested": (n, lambda r, t: oracle.sobol_points(C, 0, r, nested, sd, threads=t)),
            "sobol32_nested_from_index_1": (n, lambda r, t: oracle.sobol_points(C, 1, r, nested, sd, threads=t)),
            "sobol40_nested": (n, lambda r, t: oracle.sobol_points(C40, 0, r, nested, sd40, threads=t)),
            "sobol64_nested_at_2^40": (n, lambda r, t: oracle.sobol_points_wide(W[:s], 1 << 40, r, nested, sd,
                                                                                threads=t)),
            "sobol64_partition_p5_of_8": (n, lambda r, t: oracle.sobol_points_partitioned(W, 3, 5, 1 << 37, r, nested,
                                                                                          sd, threads=t)),
            "lattice_shifted": (nb, lambda r, t: oracle.lattice_points(g, sh, 0, r, threads=t)),
            "lattice_shifted_from_index_1": (nb, lambda r, t: oracle.lattice_points(g, sh, 1, r, threads=t)),
            "halton_faure": (nl, lambda r, t: oracle.halton_points(s, 0, r, oracle.HALTON_FAURE, threads=t)),
            "halton_faure_partition_p5_of_8": (n, lambda r, t: oracle.halton_points_partitioned(
                s, 3, 5, 1 << 30, r, oracle.HALTON_FAURE, threads=t)),
            "pixel_lattice_16spp": (8 * nl, lambda r, t: oracle.pixel_lattice_points(g, 1024, r // 16, 16,
                                                                                     height=1024)),
            "random_lattice_hash_x4_16spp": (nb, lambda r, t: oracle.random_lattice_points(
                oracle.RLAT_HASH, 7, 4, s, 1024, r // 16, 16, threads=t)),
            "random_lattice_lfsr_x4_16spp": (n // 4, lambda r, t: oracle.random_lattice_points(
                oracle.RLAT_LFSR, 7, 4, s, 1024, r // 16, 16, threads=t)),
        }
        dims = {"sobol40_nested": 40}
        out["points"] = {name: _oracle_rates(lambda k, t, rows=rows, fn=fn: _discard(fn(rows // k, t)),
                                             rows * dims.get(name, s), "Gdims/s",
                                             f"{rows} rows x {dims.get(name, s)} dims")
                         for name, (rows, fn) in runs.items()}
    return out


def attach_cpu_baselines(extras: dict, base: dict) -> None:
    """Put each oracle figure beside the GPU figure it samples (results the oracle kept
    for an error statement stay out of the figure)."""
    for name, b in base.items():
        if name in ("lattice", "points"):
            for k, v in b.items():
                if k in extras[name]:
                    extras[name][k]["cpu_baseline"] = v
        else:
            extras[name]["cpu_baseline"] = {k: v for k, v in b.items() if not k.startswith("_")}


def gradient_errors(gpu: dict, ref: dict, theta: np.ndarray, target: np.ndarray) -> dict:
    """Errors of the GPU's estimates, gradient means J and fused gradients dtheta
    against the oracle on the same pixels (theta order w, mu, nu, sigma): the largest
    relative error of the estimates and of the non-cancelling means (w, sigma: every
    term >= 0), the largest error relative to |J| + S for the cancelling ones (mu, nu;
    S = the oracle's mean of the summed absolute values of each derivative's terms),
    and quantiles of |dtheta32 - dtheta64| / |dtheta64|."""
    e, J, g = gpu["est"], gpu["J"].astype(np.float64), gpu["dtheta"].astype(np.float64)
    e64, J64, S64 = ref["est"], ref["grad"], ref["grad_scale"]
    out = {"pixels": int(e.size), "est_max_rel": float(np.max(np.abs(e - e64) / np.abs(e64)))}
    for name, k in (("w", 0), ("sigma", 3)):
        out[f"J_{name}_max_rel"] = float(np.max(np.abs(J[:, k::4] - J64[:, k::4]) / np.abs(J64[:, k::4])))
    for name, k in (("mu", 1), ("nu", 2)):
        out[f"J_{name}_max_over_J_plus_S"] = float(np.max(np.abs(J[:, k::4] - J64[:, k::4]) /
                                                          (np.abs(J64[:, k::4]) + S64[:, k::4])))
    g64 = 2.0 * (e64 - target)[:, None] * J64
    rel = np.abs(g - g64) / np.abs(g64)
    out["dtheta_rel_quantiles"] = {q: float(np.quantile(rel, float(q))) for q in ("0.5", "0.99", "1.0")}
    return out


def _r(v, digits=4):
    return None if v is None else float(f"{v:.{digits}g}")


def compact_extras(x: dict) -> dict:
    """The figures of each extra workload that the one JSON line carries (the full record
    goes to --detail-out): rates, the roofline fractions, the oracle's rates on all host
    cores and on one core, and the errors."""
    def cpu(e):
        b = e.get("cpu_baseline")
        return None if not b else [_r(b["value"], 3), _r(b.get("value_1core"), 3)]

    def roof(rf):
        pipes = rf.get("pipes")
        return {"alg_frac": _r(rf["alg_frac"], 3), "issue_frac": _r(rf.get("frac"), 3),
                "pipes": None if pipes is None else [_r(pipes[k], 2) for k in PIPES]}

    def errs(e):
        if not e:
            return None
        q = e["dtheta_rel_quantiles"]
        return {"est": _r(e["est_max_rel"], 2), "J_w": _r(e["J_w_max_rel"], 2), "J_sigma": _r(e["J_sigma_max_rel"], 2),
                "J_mu_S": _r(e["J_mu_max_over_J_plus_S"], 2), "J_nu_S": _r(e["J_nu_max_over_J_plus_S"], 2),
                "dtheta_p50_p99_max": [_r(q["0.5"], 2), _r(q["0.99"], 2), _r(q["1.0"], 2)]}

    out = {"pipes_order": list(PIPES), "oracle_order": ["all cores", "one core"]}
    if "fwd_bwd" in x:
        f = x["fwd_bwd"]
        out["fwd_bwd"] = {"gsamples_s": _r(f["fused_gsamples_s"]), "unfused": _r(f.get("unfused_gsamples_s")),
                          **roof(f["roofline"]), "oracle": cpu(f), "err_vs_oracle": errs(f.get("errors_vs_oracle"))}
    if "batched" in x:
        f = x["batched"]
        out["batched"] = {"gsamples_s": _r(f["gsamples_s"]), **roof(f["roofline"]), "oracle": cpu(f)}
    if "lattice" in x:
        for fam in ("product_peak", "oscillatory"):
            f = x["lattice"][fam]
            out[f"lattice_{fam}"] = {"gsamples_s": _r(f["gsamples_s"]), "unfused": _r(f.get("unfused_gsamples_s")),
                                     **roof(f["roofline"]), "oracle": cpu(f)}
    if "partition" in x:
        f = x["partition"]
        out["partition"] = {"gsamples_s": _r(f["gsamples_s"]), **roof(f["roofline"]), "oracle": cpu(f),
                            "rel_err_vs_exact": _r(f["rel_err_vs_exact"], 2)}
    if "points" in x:
        out["points_gdims_s_frac_hbm"] = {k: [_r(v["gdims_s"], 3), _r(v["frac_hbm"], 2)]
                                          for k, v in x["points"].items() if isinstance(v, dict) and "gdims_s" in v}
        if "fill_reference" in x["points"]:
            out["points_fill_reference_frac_hbm"] = _r(x["points"]["fill_reference"]["frac_hbm"], 3)
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    from paper_2307_15584_gb300 import inputs

    C = oracle.sobol_matrices(S_DIMS, inputs.sobol_raw_init(S_DIMS))
    seeds = inputs.scramble_seeds(S_DIMS)
    threads = os.cpu_count() or 1
    rows = 1 << 17
    for _ in range(args.warmup):
        oracle.sobol_points(C, 0, rows, oracle.SCRAMBLE_NESTED, seeds, threads=threads)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.sobol_points(C, (k * rows) % N_POINTS, rows, oracle.SCRAMBLE_NESTED, seeds, threads=threads)
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


PARITY_NOTE = ("bit-for-bit inputs, estimates within 1e-6 relative (+1e-12 W) of the fp64 oracle on the same "
               "points: tests/test_gpu_fullsize.py, tests/test_gpu_integrate.py")


def rms_rel_err(est: np.ndarray, exact: np.ndarray) -> float:
    """Root-mean-square relative error of QMC estimates against exact integrals."""
    return float(np.sqrt(np.mean(((est - exact) / exact) ** 2)))


def genz_exact(family: str, theta: np.ndarray, s: int) -> float:
    """Closed-form integrals over [0,1]^s of the Genz test functions (theta = a[s], u[s]):
    product peak  prod_j a_j (atan(a_j (1 - u_j)) + atan(a_j u_j));
    oscillatory   Re(exp(2 pi i u_1) prod_j (exp(i a_j) - 1) / (i a_j))."""
    a = np.asarray(theta[:s], np.float64)
    u = np.asarray(theta[s:2 * s], np.float64)
    if family == "product_peak":
        return float(np.prod(a * (np.arctan(a * (1 - u)) + np.arctan(a * u))))
    z = np.exp(2j * np.pi * u[0]) * np.prod((np.exp(1j * a) - 1) / (1j * a))
    return float(z.real)


def bench_fwd_bwd(dev, steps, warmup, small, sm_mhz):
    """Config 5: 1024x1024 integrals (2^16 when small) x 4096 samples, 16 parameters each."""
    import torch

    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    stream = torch.cuda.current_stream()
    n = 1 << (16 if small else 20)
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
    tuned = B.qmc_tune_integrate(prob, n, d["c"], d["th"], est, ws, target=d["tg"], grad_theta=gth, loss=loss)
    B.qmc_tune_integrate(prob, n, d["c"], d["th"], est, ws)  # the unfused forward's own split
    tf = timed(fused, steps, warmup, stream)
    out = {"pixels": n, "samples_per_pixel": 4096, "tuned": {"chunk": tuned.chunk, "block": tuned.block}}
    out["fused_ms"] = statistics.median(tf)
    out["fused_gsamples_s"] = samples / (out["fused_ms"] * 1e-3) / 1e9
    if not small:
        tu = timed(unfused, max(2, steps // 2), 2, stream)
        out["unfused_ms"] = statistics.median(tu)
        out["unfused_gsamples_s"] = samples / (out["unfused_ms"] * 1e-3) / 1e9
        unfused()
        torch.cuda.synchronize()
        e_u, g_u = est.cpu().numpy(), gb.cpu().numpy()
    fused()
    torch.cuda.synchronize()
    e, g = est.cpu().numpy(), gth.cpu().numpy()
    out["est_rms_rel_err_vs_exact"] = rms_rel_err(e, inputs.gaussmix_target(theta))
    if not small:  # the two paths evaluate the same points: their results agree to rounding
        out["fused_vs_unfused_est_max_rel_diff"] = float(np.max(np.abs(e - e_u) / np.abs(e_u)))
        out["fused_vs_unfused_grad_max_rel_diff"] = float(np.max(np.abs(g - g_u) / np.maximum(np.abs(g_u), 1e-30)))
    out["parity"] = PARITY_NOTE
    out["roofline"] = issue_roofline(out["fused_gsamples_s"] * 1e9, "integrate_main<sobol6,nested,gaussmix,grad>",
                                     sm_mhz)
    # the first 1024 pixels' estimates, fused gradients and gradient means J (a backward with
    # an upstream gradient of 1), for the error statement against the oracle's sample
    k = 1024
    B.qmc_integrate_backward(prob, n, d["c"], d["th"], torch.ones(n, dtype=torch.float64, device=dev), gb, ws)
    torch.cuda.synchronize()
    out["_gpu_sample"] = {"est": e[:k].copy(), "dtheta": g[:k].copy(), "J": gb[:k].cpu().numpy(),
                          "theta": theta[:k], "target": target[:k]}
    return out


def bench_batched(dev, steps, warmup, small, sm_mhz):
    """Config 4: 1920x1080 integrals (480x270 when small), log-uniform counts in [1, 65536]."""
    import torch

    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    stream = torch.cuda.current_stream()
    n = 480 * 270 if small else 1920 * 1080
    counts = inputs.log_uniform_counts(n)
    C6 = B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6))
    theta = inputs.gaussmix_theta(n, seed=7)
    seeds = inputs.pixel_seeds(n, 6, seed=7)
    d = {"C": B.u32_tensor(C6, dev), "c": B.u32_tensor(counts, dev), "th": torch.from_numpy(theta).to(dev),
         "sd": B.u32_tensor(seeds, dev)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"], seeds=d["sd"],
                          seeds_per_integral=True)
    ws = B.alloc_workspace(prob, n, counts, dev)
    est = torch.empty(n, dtype=torch.float64, device=dev)

    tuned = B.qmc_tune_integrate(prob, n, d["c"], d["th"], est, ws)
    # the whole batch (scans, persistent kernel, reduction) as one CUDA graph
    side = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        B.qmc_graph_begin(side)
        B.qmc_integrate(prob, n, d["c"], d["th"], est, ws, stream=side)
        graph = B.qmc_graph_end(side)

    def batched():
        B.qmc_graph_launch(graph, stream)

    tb = timed(batched, steps, warmup, stream)
    batched()
    torch.cuda.synchronize()
    B.qmc_graph_destroy(graph)
    ms = statistics.median(tb)
    gs = float(counts.sum()) / (ms * 1e-3) / 1e9
    return {"pixels": n, "samples": int(counts.sum()), "ms": ms, "gsamples_s": gs, "graph": True,
            "tuned": {"chunk": tuned.chunk, "block": tuned.block},
            "est_rms_rel_err_vs_exact": rms_rel_err(est.cpu().numpy(), inputs.gaussmix_target(theta)),
            "parity": PARITY_NOTE,
            "roofline": issue_roofline(gs * 1e9, "integrate_main<sobol6,nested,gaussmix>", sm_mhz)}


def bench_lattice(dev, steps, warmup, small, sm_mhz):
    """Config 3: rank-1 lattice s = 16, 2^26 points (2^22 when small) with CP shift, Genz
    product peak and oscillatory, 4 seeded parameter sets each; fused, and unfused
    through materialised fp32 points."""
    import torch

    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    stream = torch.cuda.current_stream()
    s, N = 16, 1 << (22 if small else 26)
    g, sh = inputs.lattice_generator(s), inputs.lattice_shift(s)
    gd, shd = B.u32_tensor(g, dev), B.u32_tensor(sh, dev)
    pts = None if small else torch.empty((N, s), dtype=torch.float32, device=dev)
    res = {"points": N, "s": s}
    for fam, kind in (("product_peak", B.F_GENZ_PRODUCT_PEAK), ("oscillatory", B.F_GENZ_OSCILLATORY)):
        theta = np.stack([inputs.genz_params(fam, s, k) for k in range(4)])
        counts = np.full(4, N, np.uint32)
        cd, thd = B.u32_tensor(counts, dev), torch.from_numpy(theta).to(dev)
        prob = B.make_problem(B.SOURCE_LATTICE, kind, s, 0, g=gd, seeds=shd)
        ws = B.alloc_workspace(prob, 4, counts, dev)
        est = torch.empty(4, dtype=torch.float64, device=dev)
        tuned = B.qmc_tune_integrate(prob, 4, cd, thd, est, ws)
        tl = timed(lambda: B.qmc_integrate(prob, 4, cd, thd, est, ws), steps, warmup, stream)
        e = est.cpu().numpy()
        exact = np.array([genz_exact(fam, t, s) for t in theta])
        ms = statistics.median(tl)
        gs = 4.0 * N / (ms * 1e-3) / 1e9
        entry = {"ms": ms, "gsamples_s": gs, "tuned": {"chunk": tuned.chunk, "block": tuned.block},
                 "rel_err_vs_exact": [float(v) for v in np.abs(e - exact) / np.abs(exact)],
                 "roofline": issue_roofline(gs * 1e9, f"integrate_main<lattice16,{fam}>", sm_mhz)}
        if pts is not None:
            est_u = torch.empty(4, dtype=torch.float64, device=dev)

            def unfused():
                B.qmc_lattice_points(gd, shd, s, 0, N, 0, None, pts)
                B.qmc_integrate_points(prob, 4, cd, pts, 1, thd, est_u, ws)

            tu = timed(unfused, max(2, steps // 2), 2, stream)
            entry["unfused_ms"] = statistics.median(tu)
            entry["unfused_gsamples_s"] = 4.0 * N / (entry["unfused_ms"] * 1e-3) / 1e9
            entry["unfused_equals_fused"] = bool(torch.equal(est_u, est))
        res[fam] = entry
    return res


def bench_points(dev, steps, warmup, small, sm_mhz):
    """Every materialising generator on the headline's shape (s = 32, 2^24 rows,
    u32 + fp32, 8 B written per coordinate; 2^20 rows when small): the 32-bit
    Sobol' headline kernel again, the same from index 1 (its first group cut by
    the range), Sobol' at s = 40 (16-byte groups of 5 chunks per lane do not fit
    the fast path: the walking kernel), Sobol' with 64-bit indices at 2^40 (Alg. 3),
    the shifted rank-1 lattice from index 1 (the flat-chunk kernel),
    one element of a partitioned Sobol' sequence (Sec. 2.5.1), the shifted
    rank-1 lattice, Halton (Faure; whole, and one element of the sequence
    partitioned by its base-2 dimension), the pixel-shifted lattice and the per-pixel
    random lattices with 4 superimposed instances (2^20 pixels x 16 samples).
    Each against the measured copy bandwidth."""
    import torch

    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    stream = torch.cuda.current_stream()
    s, n = S_DIMS, 1 << (20 if small else 24)
    peak = measured_peaks()["hbm_gbs"]
    u = torch.empty((n, s), dtype=torch.int32, device=dev)
    f = torch.empty((n, s), dtype=torch.float32, device=dev)
    C = B.u32_tensor(B.qmc_sobol_matrices(s, inputs.sobol_raw_init(s)), dev)
    W = B.u32_tensor(B.qmc_sobol_matrices_wide(s + 1, 64, inputs.sobol_raw_init(s + 1)), dev)
    sd = B.u32_tensor(inputs.scramble_seeds(s), dev)
    g, sh = B.u32_tensor(inputs.lattice_generator(s), dev), B.u32_tensor(inputs.lattice_shift(s), dev)
    s40 = 40  # the walking kernel's workload: 40 = 8 x 5, five 16-byte chunks per lane in a group
    C40 = B.u32_tensor(B.qmc_sobol_matrices(37, inputs.sobol_raw_init(37)), dev)
    C40 = torch.cat([C40, C40[:s40 - 37]])  # dimensions 37-39 reuse columns: any matrices are valid input
    sd40 = B.u32_tensor(inputs.scramble_seeds(s40), dev)
    u40 = torch.empty((n, s40), dtype=torch.int32, device=dev)
    f40 = torch.empty((n, s40), dtype=torch.float32, device=dev)
    runs = {
        "sobol32_nested": lambda: B.qmc_sobol_points(C, s, 0, n, B.SCRAMBLE_NESTED, sd, u, f),
        "sobol32_nested_from_index_1": lambda: B.qmc_sobol_points(C, s, 1, n, B.SCRAMBLE_NESTED, sd, u, f),
        "sobol40_nested": (lambda: B.qmc_sobol_points(C40, s40, 0, n, B.SCRAMBLE_NESTED, sd40, u40, f40), s40),
        "sobol64_nested_at_2^40": lambda: B.qmc_sobol_points_wide(W, 64, s, 1 << 40, n, B.SCRAMBLE_NESTED, sd, u, f),
        "sobol64_partition_p5_of_8": lambda: B.qmc_sobol_points_partitioned(W, 64, s, 3, 5, 1 << 37, n,
                                                                            B.SCRAMBLE_NESTED, sd, u, f),
        "lattice_shifted": lambda: B.qmc_lattice_points(g, sh, s, 0, n, 0, u, f),
        "lattice_shifted_from_index_1": lambda: B.qmc_lattice_points(g, sh, s, 1, n, 0, u, f),
        "halton_faure": lambda: B.qmc_halton_points(s, B.HALTON_FAURE, None, 0, n, u, f),
        "halton_faure_partition_p5_of_8": lambda: B.qmc_halton_points_partitioned(s, B.HALTON_FAURE, None, 3, 5,
                                                                                  1 << 30, n, u, f),
        "pixel_lattice_16spp": lambda: B.qmc_pixel_lattice_points(g, s, 1024, n // 16 // 1024 or 1, 0,
                                                                   n // 16, 16, u, f),
        "random_lattice_hash_x4_16spp": lambda: B.qmc_random_lattice_points(B.RLAT_HASH, 7, 4, s, 1024,
                                                                            n // 16 // 1024 or 1, 0, n // 16, 16,
                                                                            u, f),
        "random_lattice_lfsr_x4_16spp": lambda: B.qmc_random_lattice_points(B.RLAT_LFSR, 7, 4, s, 1024,
                                                                            n // 16 // 1024 or 1, 0, n // 16, 16,
                                                                            u, f),
    }
    # instruction counts per coordinate (ncu, profiles/inst_per_coord.txt) for the issue roofline
    clock = sm_mhz or measured_peaks()["sm_max_mhz"]
    issue_peak = SMS * SCHEDULERS_PER_SM * WARP * clock * 1e6  # thread-instructions/s
    res = {"rows": n, "s": s, "bytes_per_launch": n * s * 8,
           "issue_peak_ginst_s": issue_peak / 1e9, "clock_mhz": clock}
    for name, fn in runs.items():
        fn, si = fn if isinstance(fn, tuple) else (fn, s)
        ms = statistics.median(timed(fn, steps, warmup, stream))
        gbs = n * si * 8 / (ms * 1e-3) / 1e9
        entry = {"ms": ms, "gdims_s": n * si / (ms * 1e-3) / 1e9, "gb_s": gbs, "frac_hbm": gbs / peak}
        if si != s:
            entry["s"] = si
        if name in POINTS_KERNELS:
            key = POINTS_KERNELS[name][0]
            ipc = _profile_value("inst_per_coord.txt", key, profile_sources("inst_per_coord.txt", key))
            if ipc is not None:
                entry["inst_per_coord"] = ipc
                entry["frac_issue"] = ipc * n * si / (ms * 1e-3) / issue_peak
                entry["bound"] = "hbm" if entry["frac_hbm"] >= entry["frac_issue"] else "alu"
        res[name] = entry
    # context for fractions above 1: the copy peak moves every byte twice (a read and a write);
    # a write-only stream of the same two outputs by the library's fill kernels, timed the same way
    ms = statistics.median(timed(lambda: (u.fill_(0), f.fill_(0.0)), steps, warmup, stream))
    gbs = n * s * 8 / (ms * 1e-3) / 1e9
    res["fill_reference"] = {"ms": ms, "gb_s": gbs, "frac_hbm": gbs / peak, "kind": "library fill (write-only)"}
    del u, f, u40, f40
    return res


def error_spectrum_low_ratio(err: np.ndarray, band: float = 0.125) -> float:
    """Mean power of the error image below `band` cycles/pixel (radially, DC
    excluded) over its mean power at all frequencies: 1 for white noise, below 1
    when the error is pushed to high frequencies (blue-noise-like), above 1 when
    neighbouring pixels err alike."""
    e = err - err.mean()
    P = np.abs(np.fft.fft2(e)) ** 2
    fy = np.fft.fftfreq(e.shape[0])[:, None]
    fx = np.fft.fftfreq(e.shape[1])[None, :]
    r = np.sqrt(fx * fx + fy * fy)
    low = (r > 0) & (r < band)
    return float(P[low].mean() / P[r > 0].mean())


def bench_partition(dev, steps, warmup, small, sm_mhz):
    """One integral over the first 16 (2^32 - 1) ~ 6.9e10 points of a 64-bit Sobol'
    sequence (Sec. 2.5.1): the 16 elements of the sequence partitioned by its
    dimension 0 integrate as 16 integrals of 2^32 - 1 samples each (2^24 when
    small), whose mean is the estimate; Genz product peak, s = 16, nested
    scramble, with the error against the closed form."""
    import torch

    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    stream = torch.cuda.current_stream()
    s, q = 16, 4
    P, n = 1 << q, (1 << 24) if small else (1 << 32) - 1
    W = B.qmc_sobol_matrices_wide(s + 1, 64, inputs.sobol_raw_init(s + 1))
    th = inputs.genz_params("product_peak", s, 0)
    counts = np.full(P, n, np.uint32)
    d = {"W": B.u32_tensor(W, dev), "sd": B.u32_tensor(inputs.scramble_seeds(s), dev),
         "c": B.u32_tensor(counts, dev), "th": torch.from_numpy(np.tile(th, (P, 1))).to(dev)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GENZ_PRODUCT_PEAK, s, B.SCRAMBLE_NESTED, matrices=d["W"], seeds=d["sd"],
                          index_bits=64, partition_log2=q)
    ws = B.alloc_workspace(prob, P, counts, dev)
    est = torch.empty(P, dtype=torch.float64, device=dev)
    tuned = B.qmc_tune_integrate(prob, P, d["c"], d["th"], est, ws)
    ms = statistics.median(timed(lambda: B.qmc_integrate(prob, P, d["c"], d["th"], est, ws), steps, warmup, stream))
    e = est.cpu().numpy()
    exact = genz_exact("product_peak", th, s)
    samples = float(counts.sum())
    return {"elements": P, "samples_per_element": n, "samples": int(samples), "index_bits": 64, "ms": ms,
            "gsamples_s": samples / (ms * 1e-3) / 1e9, "tuned": {"chunk": tuned.chunk, "block": tuned.block},
            "estimate": float(e.mean()), "rel_err_vs_exact": float(abs(e.mean() - exact) / exact),
            "element_rel_spread": float((e.max() - e.min()) / exact), "parity": PARITY_NOTE,
            "roofline": issue_roofline(samples / (ms * 1e-3), "integrate_main<sobol16,nested,product_peak>", sm_mhz)}


def bench_samplers(dev, steps, warmup, small, sm_mhz):
    """Fig. 1 substitute (Sec. 3): two 1920x1080 images (480x270 when small),
    estimated at 4 / 16 / 64 / 256 samples per pixel by the samplers the paper
    compares, all through the fused integrator: nested-scrambled Sobol' with
    per-pixel seeds (and, on the first image, one seed vector shared by every
    pixel), the pixel-shifted rank-1 lattice (Eq. (PixelShiftedR1LS)), and
    per-pixel random lattices (Alg. 4) with hashed generator vectors, one or four
    superimposed instances, and LFSR generator vectors with four instances.
    Image one: 6-D Gaussian mixtures varying smoothly over the image (errors
    against the closed forms).  Image two: a procedural scene with checker edges
    and a soft shadow (errors against a 16384-spp reference).  Per sampler and
    rate: the RMS error, the low-frequency share of the error image's power
    spectrum, and the time."""
    import torch

    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    stream = torch.cuda.current_stream()
    W, H = (480, 270) if small else (1920, 1080)
    n = W * H
    theta = inputs.gaussmix_theta_image(W, H)
    exact = inputs.gaussmix_target(theta)
    thd = torch.from_numpy(theta).to(dev)
    C6 = B.u32_tensor(B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6)), dev)
    per_pixel = B.u32_tensor(inputs.pixel_seeds(n, 6), dev)
    shared = B.u32_tensor(inputs.scramble_seeds(6), dev)
    g = B.u32_tensor(inputs.lattice_generator(6), dev)
    seed = B.u32_tensor(np.array([inputs.DEFAULT_SEED], np.uint32), dev)
    F = B.F_GAUSSMIX4_6D
    problems = {
        "sobol_nested_per_pixel": B.make_problem(B.SOURCE_SOBOL, F, 6, B.SCRAMBLE_NESTED, matrices=C6,
                                                 seeds=per_pixel, seeds_per_integral=True),
        "sobol_nested_shared": B.make_problem(B.SOURCE_SOBOL, F, 6, B.SCRAMBLE_NESTED, matrices=C6, seeds=shared),
        "pixel_shifted_lattice": B.make_problem(B.SOURCE_PIXEL_LATTICE, F, 6, 0, g=g, image_width=W),
        "random_lattice_hash": B.make_problem(B.SOURCE_RANDOM_LATTICE, F, 6, B.rlat_randomize(B.RLAT_HASH, 1),
                                              seeds=seed, image_width=W),
        "random_lattice_hash_x4": B.make_problem(B.SOURCE_RANDOM_LATTICE, F, 6, B.rlat_randomize(B.RLAT_HASH, 4),
                                                 seeds=seed, image_width=W),
        "random_lattice_lfsr_x4": B.make_problem(B.SOURCE_RANDOM_LATTICE, F, 6, B.rlat_randomize(B.RLAT_LFSR, 4),
                                                 seeds=seed, image_width=W),
    }
    est = torch.empty(n, dtype=torch.float64, device=dev)

    def compare(problems, theta_d, reference, relative):
        out = {}
        for name, prob in problems.items():
            entry = {"rms_err": [], "low_freq_ratio": [], "ms": []}
            for spp in (4, 16, 64, 256):
                counts = np.full(n, spp, np.uint32)
                cd = B.u32_tensor(counts, dev)
                ws = B.alloc_workspace(prob, n, counts, dev)
                ms = statistics.median(timed(lambda: B.qmc_integrate(prob, n, cd, theta_d, est, ws), steps, warmup,
                                             stream))
                diff = est.cpu().numpy() - reference
                err = (diff / reference if relative else diff / np.abs(reference).mean()).reshape(H, W)
                entry["rms_err"].append(float(np.sqrt(np.mean(err * err))))
                entry["low_freq_ratio"].append(error_spectrum_low_ratio(err))
                entry["ms"].append(ms)
                del ws
            entry["gsamples_s_at_256spp"] = n * 256 / (entry["ms"][-1] * 1e-3) / 1e9
            out[name] = entry
        return out

    res = {"image": [W, H], "spp": [4, 16, 64, 256],
           "metrics": "rms_err; low_freq_ratio = error power below 1/8 cycle/pixel over mean power (white noise 1)"}
    res["mixture"] = {"integrand": "gaussmix, smooth over the image", "reference": "closed form",
                      "error": "relative per pixel", **compare(problems, thd, exact, True)}

    # the procedural scene: discontinuous (checker edges, the shadow of a sphere), no closed form;
    # the reference is per-pixel nested-scrambled Sobol' at 16384 samples per pixel
    theta_s = torch.from_numpy(inputs.scene_theta(W, H)).to(dev)
    C4 = B.u32_tensor(B.qmc_sobol_matrices(4, inputs.sobol_raw_init(4)), dev)
    pp4 = B.u32_tensor(inputs.pixel_seeds(n, 4), dev)
    g4 = B.u32_tensor(inputs.lattice_generator(4), dev)
    Fs = B.F_SCENE4D
    ref_prob = B.make_problem(B.SOURCE_SOBOL, Fs, 4, B.SCRAMBLE_NESTED, matrices=C4,
                              seeds=B.u32_tensor(inputs.pixel_seeds(n, 4, seed=inputs.DEFAULT_SEED + 7), dev),
                              seeds_per_integral=True)
    ref_counts = np.full(n, 1 << 14, np.uint32)
    ref_ws = B.alloc_workspace(ref_prob, n, ref_counts, dev)
    B.qmc_integrate(ref_prob, n, B.u32_tensor(ref_counts, dev), theta_s, est, ref_ws)
    reference = est.cpu().numpy().copy()
    del ref_ws
    scene = {
        "sobol_nested_per_pixel": B.make_problem(B.SOURCE_SOBOL, Fs, 4, B.SCRAMBLE_NESTED, matrices=C4, seeds=pp4,
                                                 seeds_per_integral=True),
        "pixel_shifted_lattice": B.make_problem(B.SOURCE_PIXEL_LATTICE, Fs, 4, 0, g=g4, image_width=W),
        "random_lattice_hash": B.make_problem(B.SOURCE_RANDOM_LATTICE, Fs, 4, B.rlat_randomize(B.RLAT_HASH, 1),
                                              seeds=seed, image_width=W),
        "random_lattice_hash_x4": B.make_problem(B.SOURCE_RANDOM_LATTICE, Fs, 4, B.rlat_randomize(B.RLAT_HASH, 4),
                                                 seeds=seed, image_width=W),
        "random_lattice_lfsr_x4": B.make_problem(B.SOURCE_RANDOM_LATTICE, Fs, 4, B.rlat_randomize(B.RLAT_LFSR, 4),
                                                 seeds=seed, image_width=W),
    }
    res["scene"] = {"integrand": "checkerboard under a square light, shadow of a sphere (discontinuous)",
                    "reference": "nested-scrambled Sobol', 16384 spp per pixel",
                    "error": "per pixel, relative to the image's mean", **compare(scene, theta_s, reference, False)}
    return res


def run_extras(args, dev, sm_mhz):
    which = [args.only] if args.only else ["fwd_bwd", "batched", "lattice", "points", "partition"]
    fns = {"fwd_bwd": bench_fwd_bwd, "batched": bench_batched, "lattice": bench_lattice,
           "points": bench_points, "samplers": bench_samplers, "partition": bench_partition}
    out = {}
    for name in which:
        steps = 3 if args.small else 5
        out[name] = fns[name](dev, steps, 3, args.small, sm_mhz)
        import torch

        torch.cuda.empty_cache()
    return out


def finish_extras(extras: dict, with_cpu: bool) -> None:
    """The oracle's samples beside the GPU figures, and the fused gradient's errors
    against the oracle's results on its sample of pixels."""
    base = extras_cpu_baselines(list(extras)) if with_cpu else {}
    fb = extras.get("fwd_bwd")
    if fb is not None:
        gpu = fb.pop("_gpu_sample", None)
        ref = base.get("fwd_bwd", {}).get("_result")
        if gpu is not None and ref is not None:
            fb["errors_vs_oracle"] = gradient_errors(gpu, ref, gpu["theta"], gpu["target"])
    attach_cpu_baselines(extras, base)


def write_detail(path, record) -> None:
    if path:
        with open(path, "w") as f:
            json.dump(record, f, indent=1)


def run_ours(args, world, rank, local):
    import torch

    from paper_2307_15584_gb300 import binding as B
    from paper_2307_15584_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.only:  # one integration workload alone (profiling); no headline line
        res = run_extras(args, dev, None)
        finish_extras(res, not args.no_cpu)
        write_detail(args.detail_out, res)
        print(json.dumps({"only": args.only, "small": args.small, **res}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()

    begin, count = rank_window(rank, world, 1 << args.log2_points)
    seeds = inputs.scramble_seeds(S_DIMS)
    if args.plan == "window":
        C = B.qmc_sobol_matrices(S_DIMS, inputs.sobol_raw_init(S_DIMS))
    else:  # dimensions 1..s of the wide matrices; dimension 0 selects the rank's element
        q, p = rank_partition(rank, world)
        C = B.qmc_sobol_matrices_wide(S_DIMS + 1, 64, inputs.sobol_raw_init(S_DIMS + 1))
    Cd, sd = B.u32_tensor(C, dev), B.u32_tensor(seeds, dev)
    out_u = torch.empty((count, S_DIMS), dtype=torch.int32, device=dev)
    out_f = torch.empty((count, S_DIMS), dtype=torch.float32, device=dev)

    def launch(u, f):
        if args.plan == "window":
            B.qmc_sobol_points(Cd, S_DIMS, begin, count, B.SCRAMBLE_NESTED, sd, u, f)
        else:
            B.qmc_sobol_points_partitioned(Cd, 64, S_DIMS, q, p, 0, count, B.SCRAMBLE_NESTED, sd, u, f)

    def step():
        launch(out_u, out_f)

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

    def e2e_direct():  # the kernel writes the points straight into pinned host memory (NVLink-C2C)
        Cd.copy_(h_C, non_blocking=True)
        sd.copy_(h_s, non_blocking=True)
        launch(h_u.data_ptr(), h_f.data_ptr())

    def d2h_only():  # the host link alone: the same bytes copied without the kernel
        h_u.copy_(out_u, non_blocking=True)
        h_f.copy_(out_f, non_blocking=True)

    e2e_copy_ms = statistics.median(timed(e2e_step, 3, 1, stream))
    e2e_direct_ms = statistics.median(timed(e2e_direct, 3, 1, stream))
    link_ms = statistics.median(timed(d2h_only, 3, 1, stream))
    e2e_ms = min(e2e_copy_ms, e2e_direct_ms)
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
        "config": {"workload": f"materialised scrambled Sobol': s={S_DIMS}, {count} indices per GPU, nested "
                               f"scramble, u32 + f32 outputs [{count}][{S_DIMS}]", "s": S_DIMS,
                   "points_per_gpu": count, "scramble": "nested", "outputs": "u32+f32",
                   "plan": ("index window per GPU" if args.plan == "window"
                            else f"element {rank} of P = {world} of the sequence partitioned by its phi_2 "
                                 "dimension"),
                   "l2": "4 GiB of outputs per step > 129 MB L2: no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": profile_traffic("sobol_points_fast<1,2>"),
                     "peak_source": peaks["source"] + " copy",
                     "algorithmic_bytes_per_launch": bytes_per_launch},
        "e2e": {"value": coords / (e2e_ms * 1e-3) / 1e9, "unit": "Gdims/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "method": "kernel writes pinned host" if e2e_direct_ms <= e2e_copy_ms else "device + copy to host",
                "link_gbs": d2h / (link_ms * 1e-3) / 1e9, "link_frac": (link_ms / e2e_ms)},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    e2e_detail = {"ms_copy_back": e2e_copy_ms, "ms_direct_to_host": e2e_direct_ms, "ms_link_alone": link_ms,
                  "achieved_gbs": (h2d + d2h) / (e2e_ms * 1e-3) / 1e9}
    del out_u, out_f, h_u, h_f
    torch.cuda.empty_cache()
    extras = run_extras(args, dev, clk.get("sm_mhz")) if not args.no_extra else None
    if not args.no_cpu:
        cb = cpu_baseline()
        line["cpu_baseline"] = {k: v for k, v in cb.items() if k in ("value", "unit", "cores", "kind", "value_1core")}
        line["cpu_baseline"]["sample"] = f"2^23 of the 2^24 points (1/16 of that on one core)"
    if extras is not None:
        finish_extras(extras, not args.no_cpu)
        write_detail(args.detail_out, {"line": line, "e2e_detail": e2e_detail, "extras": extras})
        line["fused"] = compact_extras(extras)  # last, so that the end of the output holds it
    print(json.dumps(line, separators=(",", ":")), flush=True)
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
