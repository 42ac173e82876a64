#!/usr/bin/env python
"""Benchmark of the hybrid DM-baryon interaction step on GB300.

One step = the whole hot path on one synthetic galaxy: Morton grid, pair search in both
directions, gas mean field, DM Monte Carlo, kicks and float64 sums (dmb_step through the
C ABI).  Workload: 8M DM in a Hernquist halo + 2M gas in an exponential disk
(`galaxy10M`), sigma = sigma0 (v/100 km/s)^n.

Metric: DM-gas pair interactions per second (pairs of the step / step time); the line also
reports particles stepped per second.  `value` is device-resident throughput (inputs in
HBM); `e2e` repeats the step through the same C ABI with the inputs copied from pinned
host memory and the results copied back inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dmb|reference] [--n 0]

--impl reference times the FP64 oracle (the method's plain CPU restatement) on bounded
spatial samples of the same workload.  Under torchrun every rank runs an independent
replica (the step does not shard across GPUs in this build).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# measured on this GPU model (152 SMs, 128 FP32 lanes per SM): lane operations per clock
SMS = 152
LANES = 128
# algorithmic lane operations per pair (FMA = 1 op, special functions = 1 op), counted from
# the formulas each kernel evaluates: the overlap table lookup, the pair geometry, the 1F1
# rates and the float64-free sums for the mean field; Philox, Box-Muller, the overlap and the
# fixed-point running sum for the Monte Carlo
OPS_PER_PAIR = {"meanfield": 150.0, "mc": 256.0}
# of those, the pair's geometry (split-float displacement, distance, the overlap table's bicubic
# lookup, M_i g); a float32 search with pair weights (dmb_set_pair_weights) evaluates it once per
# pair in its emit pass and the mean field and the Monte Carlo read the stored weights
GEOM_OPS_PER_PAIR = 84.0
OPS_PER_PAIR_F32 = {k: v - GEOM_OPS_PER_PAIR for k, v in OPS_PER_PAIR.items()}
# of the mean field's 150, the closed-form rates (1F1 by its recurrence: one exp, one erf, ~40 FMA);
# with the surrogate or the quadrature the pass reads or computes its rates otherwise
RATE_OPS_CLOSED = 42.0
# the float32 mean-field kernel's algorithmic bytes per pair with stored weights: row index,
# weight, the DM velocity copy, and the pair's (FA, FB) with the surrogate
MF_BYTES_PER_PAIR = {"closed": 4 + 4 + 16.0, "quad": 4 + 4 + 16.0, "mlp": 4 + 4 + 16 + 8.0}
# pair search: lane operations per candidate test of the tile stage's count pass (the split-float
# displacement with the minimum image, the squared distance and the strict comparison with
# h_i + h_j, the ballots and the mask bookkeeping)
SEARCH_OPS_PER_TEST = 25.0
# quadrature provider: 64 nodes x (2 exp + ~14 ops) + the 120 ops of the rest of the pair
QUAD_OPS_PER_PAIR = 64 * 16 + 120.0
# learned surrogate per pair: the network's dense contraction, 2 x (4 x 128 + 2 x 128 x 128 +
# 128 x 2) flop (bf16 tensor cores for the 128-wide layers), and the flop the tensor cores issue
# for it: 2 x 128 x (16 + 128 + 16 + 128 + 16) (layer 1 and its bias as one K = 16 hi/lo product,
# one K = 16 bias slice for each of layers 2 and 3).  The squared-ReLU epilogue needs no special function.
MLP_FLOP_PER_PAIR = 2.0 * (4 * 128 + 2 * 128 * 128 + 128 * 2)
MLP_TENSOR_FLOP_PER_PAIR = 2.0 * 128 * (16 + 128 + 16 + 128 + 16)
# DRAM bytes per pair of the surrogate pass from one ncu capture of the current kernel on galaxy1M
# (dram__bytes_read.sum + dram__bytes_write.sum = 712.3 + 639.2 MB for 85,071,169 pairs), scaled
# to a launch by its pair count.  Algorithmic bytes: row index, DM index, two 16-byte velocity
# copies read and the 8-byte rates written per pair
MLP_DRAM_BYTES_PER_PAIR = (712.270e6 + 639.172864e6) / 85071169
MLP_ALGO_BYTES_PER_PAIR = 4 + 4 + 16 + 16 + 8
# The same kernel with the mean field in its epilogue (--surrogate-epilogue 1): its DRAM bytes
# per pair from one ncu capture on galaxy1M (dram__bytes_read.sum + dram__bytes_write.sum =
# 782.1 + 82.9 MB for 85,071,169 pairs).
# Algorithmic bytes: row index, DM index, the two velocity copies and the two position copies
# (hi, lo) of both particles read per pair, one 24-byte partial sum written per 32 pairs
MLP_MF_DRAM_BYTES_PER_PAIR = (782.105856e6 + 82.870272e6) / 85071169
MLP_MF_ALGO_BYTES_PER_PAIR = 4 + 4 + 6 * 16 + 24 / 32
# the surrogate's training recipe (samples of the float64 device quadrature, Adam epochs)
TRAIN = dict(nsamples=1 << 21, epochs=128, seed=11)
# the power-law indices of the benchmark's cross-section scan
SCAN_N = (-4, -2, 0, 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dmb", choices=["dmb", "reference"])
    ap.add_argument("--workload", default="galaxy10M")
    ap.add_argument("--n", type=int, default=-2, help="power-law index of sigma(v) = sigma0 (v/100 km/s)^n")
    ap.add_argument("--rate", default="mlp", choices=["mlp", "quad", "closed"],
                    help="rate provider of the timed step (the others are timed beside it)")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other rate providers")
    ap.add_argument("--pair-weights", type=int, default=-1, choices=[-1, 0, 1],
                    help="dmb_set_pair_weights: -1 the library's default (not for a step's own search), 0 never, 1 always")
    ap.add_argument("--surrogate-epilogue", type=int, default=0, choices=[0, 1],
                    help="1: the surrogate's tensor-core kernel sums the mean field itself; 0: it stores the rates")
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--retune", action="store_true", help="run the autotuner even if shapes are stored")
    ap.add_argument("--quick-train", action="store_true",
                    help="train the surrogate briefly (profiling runs: the pass's work does not depend on the weights)")
    ap.add_argument("--fp64", action="store_true", help="float64 pair arithmetic (the box4k configuration)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def make_workload(name, n, seed_offset=0):
    from paper_2603_24688_gb300 import workloads as W
    if name == "galaxy10M":
        return W.galaxy_workload(8_000_000, 2_000_000, seed=W.SEED_BASE + 3 + seed_offset, n=n)
    if name == "galaxy1M":
        return W.galaxy_workload(1_000_000, 1_000_000, seed=W.SEED_BASE + 2 + seed_offset, n=n)
    if name == "box4k":
        return W.box_workload(seed=W.SEED_BASE + 1 + seed_offset, n=n)
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                   parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_across_ranks(ms, pairs, dist=None):
    """Whole-job numbers: the slowest rank's time and the sum of all ranks' pairs.

    Works on any torch.distributed backend (NCCL tensors live on the GPU, gloo on CPU)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(pairs)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def cpu_oracle_sample(w, budget_s=12.0, target_pairs=150_000, seed=0):
    """Time the FP64 oracle's full step on a spatial sub-box of the workload.

    The sub-box is a cube around a random gas particle, sized so that it holds about
    target_pairs pairs; returns (pairs/s, pairs, seconds, description)."""
    from oracle.pairs import pairs_bruteforce
    from oracle.step import oracle_step
    rng = np.random.default_rng(seed)
    dm, gas = w["dm"], w["gas"]
    c = gas["pos"][rng.integers(len(gas["h"]))]
    side = 4.0 * float(np.median(gas["h"]))
    for _ in range(30):
        sd = np.all(np.abs(dm["pos"] - c) < side / 2, axis=1)
        sg = np.all(np.abs(gas["pos"] - c) < side / 2, axis=1)
        if sd.sum() * sg.sum() > 0:
            sub_dm = {k: v[sd] for k, v in dm.items()}
            sub_gas = {k: v[sg] for k, v in gas.items()}
            pi, pj = pairs_bruteforce(sub_dm, sub_gas, w["params"]["periodic"], w["params"]["box"])
            if len(pi) >= target_pairs or side > 50:
                break
        side *= 1.3
    t0 = time.perf_counter()
    out = oracle_step(sub_dm, sub_gas, w["params"], 0, w["dt"], pairs=(pi, pj))
    t = time.perf_counter() - t0
    # the pair search is part of the oracle step: time it too
    t1 = time.perf_counter()
    pairs_bruteforce(sub_dm, sub_gas, w["params"]["periodic"], w["params"]["box"])
    t += time.perf_counter() - t1
    n = len(pi)
    desc = (f"oracle_step on a {side:.3f} kpc cube of {w['name']} ({len(sub_dm['h'])} DM, "
            f"{len(sub_gas['h'])} gas, {n} pairs), single numpy thread")
    return n / t, n, t, desc


def host_cpu_count():
    """Logical CPUs listed in /proc/cpuinfo (falls back to os.cpu_count())."""
    try:
        with open("/proc/cpuinfo") as f:
            n = sum(1 for line in f if line.startswith("processor"))
        if n > 0:
            return n
    except OSError:
        pass
    return os.cpu_count() or 1


def _subcubes(w, count, target_pairs, seed):
    """`count` spatial sub-cubes of the workload around random gas particles: the first sized (by
    a brute-force pair count) to hold about target_pairs pairs, the others of the same side but
    shrunk where the region is denser, until their DM x gas particle product is at most twice the
    first cube's.  Returns the cubes and the (min, max) side."""
    from oracle.pairs import pairs_bruteforce
    rng = np.random.default_rng(seed)
    dm, gas = w["dm"], w["gas"]

    def cut(sp_dm, sp_gas, c, side):
        sd = np.all(np.abs(sp_dm["pos"] - c) < side / 2, axis=1)
        sg = np.all(np.abs(sp_gas["pos"] - c) < side / 2, axis=1)
        return {k: v[sd] for k, v in sp_dm.items()}, {k: v[sg] for k, v in sp_gas.items()}

    c = gas["pos"][rng.integers(len(gas["h"]))]
    side = 4.0 * float(np.median(gas["h"]))
    for _ in range(30):
        sub_dm, sub_gas = cut(dm, gas, c, side)
        if len(sub_dm["h"]) * len(sub_gas["h"]) > 0:
            pi, _ = pairs_bruteforce(sub_dm, sub_gas, w["params"]["periodic"], w["params"]["box"])
            if len(pi) >= target_pairs or side > 50:
                break
        side *= 1.3
    cubes = [(sub_dm, sub_gas)]
    cap = 2 * max(len(sub_dm["h"]) * len(sub_gas["h"]), 1)
    sides = [side]
    while len(cubes) < count:
        c = gas["pos"][rng.integers(len(gas["h"]))]
        s = side
        sub_dm, sub_gas = cut(dm, gas, c, s)
        while len(sub_dm["h"]) * len(sub_gas["h"]) > cap and s > 1e-4:
            s /= 1.3
            sub_dm, sub_gas = cut(sub_dm, sub_gas, c, s)
        if len(sub_dm["h"]) and len(sub_gas["h"]):
            cubes.append((sub_dm, sub_gas))
            sides.append(s)
    return cubes, (min(sides), max(sides))


def _oracle_cube_job(job):
    """One oracle step (pair search by brute force, then oracle_step) on one sub-cube; runs in a
    worker process with numpy limited to one thread."""
    from oracle.pairs import pairs_bruteforce
    from oracle.step import oracle_step
    sub_dm, sub_gas, params, dt = job
    t0 = time.perf_counter()
    pi, pj = pairs_bruteforce(sub_dm, sub_gas, params["periodic"], params["box"])
    oracle_step(sub_dm, sub_gas, params, 0, dt, pairs=(pi, pj))
    return len(pi), time.perf_counter() - t0


def _noop(_):
    return 0


def cpu_oracle_all_cores(w, target_pairs=60_000, per_core=2, seed=0, cores=None):
    """Time the FP64 oracle on all host cores: one worker process per core (spawned, numpy pinned
    to one thread each), each running oracle steps on its own spatial sub-cubes of the workload.
    Returns (pairs/s over the wall time, pairs, wall seconds, cores, description)."""
    import multiprocessing as mp
    cores = cores or host_cpu_count()
    cubes, (smin, smax) = _subcubes(w, cores * per_core, target_pairs, seed)
    jobs = [(d, g, w["params"], w["dt"]) for d, g in cubes]
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_noop, range(cores))                       # start the workers before timing
            t0 = time.perf_counter()
            res = pool.map(_oracle_cube_job, jobs, chunksize=1)
            wall = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    n = sum(r[0] for r in res)
    desc = (f"oracle_step (+ brute-force pairs) on {len(jobs)} cubes of {smin:.3f}-{smax:.3f} kpc of {w['name']} "
            f"({n} pairs in total), {cores} worker processes, one numpy thread each; wall time")
    return n / wall, n, wall, cores, desc


def envelope(n):
    """Envelopes (p, q, r, m) of the surrogate's FA and FB for sigma ~ v^n: E = (1 + p x + q x^2 +
    r x^3)^m with the large-x power of 1F1(a, b; -x) and its first two Taylor coefficients."""
    def of(a, b):
        e = -a
        if e == 0:
            return 0.0, 0.0, 0.0, 0.0
        m, k1, k2 = e / 3.0, e / b, e * (e - 1.0) / (2.0 * b * (b + 1.0))
        p = k1 / m
        return p, max((k2 - 0.5 * k1 * k1) / m + 0.5 * p * p, 0.0), (math.gamma(b) / math.gamma(b + e)) ** (1.0 / m), m
    return of(-(n + 1) / 2.0, 2.5), of(-(n + 3) / 2.0, 1.5)


def bind_to_gpu_numa_node(dev):
    """Bind this process to the CPUs of the NUMA node the GPU hangs off (sysfs), so that host
    memory it allocates from now on (first touch) is local to the GPU; returns the node or None."""
    import torch
    try:
        p = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (getattr(p, "pci_domain_id", 0), p.pci_bus_id, p.pci_device_id)
        with open(f"/sys/bus/pci/devices/{bus}/numa_node") as f:
            node = int(f.read().strip())
        if node < 0:
            return None
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return node
    except (AttributeError, OSError, ValueError, RuntimeError, AssertionError):
        return None                      # no device, no sysfs entry or no per-node CPU list


def workload_tau(w):
    """(min, max) of tau = varsigma^2 / v0^2 over the workload's hot gas, varsigma^2 = k_B T / (mu m_p)."""
    kt = 1.380649e-16 / 1.67262192e-24 / 1e10                  # k_B / m_p in (km/s)^2 / K
    T, mu = w["gas"]["T"], w["gas"]["mu"]
    hot = T > 0
    tau = kt * T[hot] / mu[hot] / w["params"]["v0_kms"] ** 2
    return float(tau.min()), float(tau.max())


def rate_errors(params, n, prm, s, tau, m):
    """Relative errors of the surrogate's FA, FB (tensor-core engine) against the float64 device
    quadrature at index n, at the inputs (s, tau, m_chi) given as flat arrays."""
    import torch
    from paper_2603_24688_gb300 import dmb
    X = np.stack([0.5 * np.log10(s), 0.5 * np.log10(tau), np.log10(m), np.full(s.size, n / 4.0)],
                 1).astype(np.float32)
    c = dmb.Context(prm["sigma0_cm2"], n, prm["m_chi_mp"], prm["v0_kms"], False, (0.0, 0.0, 0.0), prm["seed"],
                    rate_mode=dmb.DMB_RATE_MLP)
    c.dmb_load_surrogate(params)
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
    c.dmb_surrogate_infer_tc(torch.from_numpy(X).cuda(), Y)
    q = dmb.Context(prm["sigma0_cm2"], n, prm["m_chi_mp"], prm["v0_kms"], False, (0.0, 0.0, 0.0), prm["seed"],
                    fp64=True, rate_mode=dmb.DMB_RATE_QUAD)
    x = 0.5 * s.astype(np.float64) ** 2
    F = torch.empty((x.size, 2), dtype=torch.float64, device="cuda")
    q.dmb_debug_rates(torch.from_numpy(x).cuda(), F)
    torch.cuda.synchronize()
    F, Y = F.cpu().numpy(), Y.cpu().numpy().astype(np.float64)
    envA, envB = envelope(n)

    def log_env(env):
        p, q, r, m = env
        return m * np.log1p(x * (p + x * (q + x * r)))
    eA_ = np.abs(np.expm1(Y[:, 0] - (np.log(F[:, 0]) - log_env(envA))))
    eB_ = np.abs(np.expm1(Y[:, 1] - (np.log(F[:, 1]) - log_env(envB))))
    c.close()
    q.close()
    return {"mean_A": float(eA_.mean()), "max_A": float(eA_.max()), "mean_B": float(eB_.mean()),
            "max_B": float(eB_.max())}


def surrogate_errors(params, n, prm, tau=None, m_chi=None):
    """rate_errors on a grid over the training box (s: 161 points, tau: 6, m_chi: 3), or with
    tau = (lo, hi) and m_chi given, over the whole s range at the workload's own tau range (6
    points, or 1 if lo == hi) and m_chi (s: 641 points)."""
    if tau is None:
        s, taus, ms = np.geomspace(1e-2, 1e2, 161), np.geomspace(1e-3, 1e2, 6), np.array([0.5, 2.0, 10.0])
    else:
        s = np.geomspace(1e-2, 1e2, 641)
        taus = np.array([tau[0]]) if tau[0] == tau[1] else np.geomspace(tau[0], tau[1], 6)
        ms = np.array([m_chi])
    S, T, M = np.meshgrid(s, taus, ms, indexing="ij")
    return rate_errors(params, n, prm, S.ravel(), T.ravel(), M.ravel())


def workload_pair_inputs(ctx, dm, gas, prm, k=1 << 20, seed=5):
    """(s, tau) of k pairs drawn uniformly (seeded) from the pair set of (dm, gas), searched on
    the given context, hot gas only: s = |v_i - V_j| / varsigma_j, tau = varsigma_j^2 / v0^2,
    varsigma^2 = k_B T / (mu m_p)."""
    import torch
    ctx.dmb_build_grid(dm, gas)
    npairs = ctx.dmb_neighbors()
    pairs = torch.empty((npairs, 2), dtype=torch.int32, device="cuda")
    ctx.dmb_neighbors(pairs)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    idx = torch.randint(0, npairs, (k,), device="cuda", generator=g)
    pi, pj = pairs[idx, 0].long(), pairs[idx, 1].long()
    del pairs
    kt = 1.380649e-16 / 1.67262192e-24 / 1e10
    sig2 = kt * gas["T"][pj] / gas["mu"][pj]
    hot = sig2 > 0
    w = torch.linalg.norm(dm["vel"][pi] - gas["vel"][pj], dim=1)
    s = (w[hot] / torch.sqrt(sig2[hot])).cpu().numpy()
    tau = (sig2[hot] / prm["v0_kms"] ** 2).cpu().numpy()
    return s, tau


def workload_desc(a, w):
    """The config's workload string, the same for both arms."""
    nd, ng = len(w['dm']['h']), len(w['gas']['h'])
    if w["params"]["periodic"]:
        L = w["params"]["box"][0]
        geom = f"periodic {L:g} kpc box, {nd} DM + {ng} gas at uniform positions"
    else:
        geom = f"{nd} DM Hernquist halo + {ng} gas exponential disk"
    prec = ", float64 pair arithmetic" if getattr(a, "fp64", False) else ""
    return f"{a.workload}: {geom}, sigma = 1e-24 cm^2 (v / 100 km/s)^{a.n}{prec}"


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = make_workload(a.workload, a.n)
    vals = []
    cores = host_cpu_count()
    for k in range(a.warmup + a.steps):
        # one step = a bounded sample of the workload, spread over every host core
        rate, npairs, t, cores, desc = cpu_oracle_all_cores(w, target_pairs=40_000, per_core=1, seed=k,
                                                            cores=cores)
        if k >= a.warmup:
            vals.append((rate, npairs, t))
    rate = sum(v[1] for v in vals) / sum(v[2] for v in vals)
    line = {"metric": "pair_interactions_per_s", "value": rate, "unit": "pairs/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(v[2] for v in vals) / len(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_desc(a, w),
                       "rate_provider": "closed-form 1F1 (the oracle; timed on bounded spatial samples)"},
            "cpu_baseline": {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": desc, "host_cpus": host_cpu_count()},
            "e2e": {"value": rate, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_substeps(a, peaks, peak_kind):
    """Hierarchical substeps of the 32M DM + 8M gas galaxy (power-of-two timestep bins, 1-10% of
    the particles active per substep): grid and pairs once, then dmb_substep replayed from CUDA
    graphs with the learned surrogate.  One timed step = one substep."""
    import torch
    from paper_2603_24688_gb300 import dmb
    from paper_2603_24688_gb300 import workloads as W
    w = W.named("galaxy40M", n=a.n)
    prm = w["params"]
    stream = torch.cuda.current_stream()
    ctx = dmb.Context(prm["sigma0_cm2"], prm["n"], prm["m_chi_mp"], prm["v0_kms"], False, (0.0, 0.0, 0.0),
                      prm["seed"], rate_mode=dmb.DMB_RATE_MLP, stream=stream)
    ctx.dmb_set_surrogate_epilogue(a.surrogate_epilogue)
    ctx.dmb_set_pair_weights(a.pair_weights)
    rep = ctx.dmb_train_surrogate(**TRAIN)
    dm, gas = dmb.to_device(w["dm"]), dmb.to_device(w["gas"])
    db = torch.from_numpy(w["dm_bin"]).cuda()
    gb = torch.from_numpy(w["gas_bin"]).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.dmb_build_grid(dm, gas)
    npairs = ctx.dmb_neighbors()
    ctx.dmb_set_bins(db, gb)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    dt = w["dt"]
    out = {}
    first = 1                  # timed substeps 1 .. K: every bin up to nu(K) active in turn
    nus = sorted({(s & -s).bit_length() - 1 for s in range(first, first + a.steps)})
    for graph in (False, True):
        ctx.dmb_set_graph(graph)
        # warm-up: W substeps, and (graph mode) one substep of every active set the timed range
        # uses, so that every graph is captured before the timed region
        warm = list(range(first, first + a.warmup)) + ([1 << nu for nu in nus] if graph else [])
        for s in warm:
            ctx.dmb_substep(dm, gas, s, dt, want_sums=False)
        evals = act = 0
        for s in range(first, first + a.steps):
            info = ctx.dmb_substep_info(s)
            act += info[0] + info[1]
            evals += 0.5 * (info[3] + info[4])
        l0 = ctx.dmb_launch_count()
        clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]) if graph else None
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(first, first + a.steps):
            ctx.dmb_substep(dm, gas, s, dt, want_sums=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[graph] = dict(ms=ms, evals=evals, active=act, launches=ctx.dmb_launch_count() - l0,
                          clocks=clocks.stop() if clocks else None, first=first)
    g = out[True]
    line = {"metric": "pair_interactions_per_s", "value": g["evals"] / (g["ms"] * 1e-3), "unit": "pairs/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": g["ms"] / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 pairs, f64 sums",
            "data": "synthetic",
            "config": {"workload": f"galaxy40M: 32000000 DM + 8000000 gas, sigma = 3e-26 cm^2 (v/100 km/s)^{a.n}, "
                                   f"power-of-two timestep bins, substeps {g['first']}..{g['first'] + a.steps - 1} "
                                   f"(graph replay) after the grid and pairs were built once",
                       "rate_provider": "learned surrogate (tcgen05 tensor cores)", "pairs_full": npairs,
                       "l2": "state (~3 GB) larger than L2; no flush", "parallelism": "replicas x1"},
            "particles_stepped_per_s": g["active"] / (g["ms"] * 1e-3),
            "active_fraction": g["active"] / (a.steps * (len(w["dm"]["h"]) + len(w["gas"]["h"]))),
            "eager": {"ms_per_step": out[False]["ms"] / a.steps,
                      "pairs_per_s": out[False]["evals"] / (out[False]["ms"] * 1e-3)},
            "setup_s": setup_s, "pair_weights": "stored by the search (dmb_neighbors keeps the pair set)"
            if a.pair_weights != 0 else "none", "gpu_launches": int(g["launches"]), "clocks": g["clocks"],
            "surrogate_val_mean_rel_err": [float(rep[3]), float(rep[4])], "peak_kind": peak_kind}
    print(json.dumps(line))
    ctx.close()
    return 0


def run_boxes(a, peaks, peak_kind):
    """The batched parameter scan: 64 independent periodic boxes (particle counts, sigma0, m_chi
    and T drawn per box) stepped together by dmb_step_batched; one timed step = one batched step
    (grid, pairs, mean field, Monte Carlo, kicks of all boxes)."""
    import torch
    from paper_2603_24688_gb300 import dmb
    from paper_2603_24688_gb300 import workloads as W
    w = W.boxes_workload(n=a.n)
    prm = w["params"]
    stream = torch.cuda.current_stream()
    ctx = dmb.Context(prm["sigma0_cm2"], prm["n"], prm["m_chi_mp"], prm["v0_kms"], True, tuple(prm["box"]),
                      prm["seed"], stream=stream)
    ctx.dmb_set_pair_weights(a.pair_weights)
    dm, gas = dmb.to_device(w["dm"]), dmb.to_device(w["gas"])
    dbx = torch.from_numpy(w["dm_box"].view(np.int32)).cuda()
    gbx = torch.from_numpy(w["gas_box"].view(np.int32)).cuda()
    step = 0
    sums = None
    # the direct launches first (stage times), then the captured step
    ctx.dmb_set_timing(True)
    for _ in range(2):
        ctx.dmb_step_batched(dm, dbx, gas, gbx, w["boxes"], step, w["dt"], want_sums=False)
        step += 1
    stage_ms, nsteps = ctx.dmb_stage_times()
    ctx.dmb_set_timing(False)
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(2):
        ctx.dmb_step_batched(dm, dbx, gas, gbx, w["boxes"], step, w["dt"], want_sums=False)
        step += 1
    d1.record(stream)
    torch.cuda.synchronize()
    direct_ms = d0.elapsed_time(d1) / 2
    ctx.dmb_set_graph(True)
    for _ in range(a.warmup):         # the first captures the step, the others replay it
        sums = ctx.dmb_step_batched(dm, dbx, gas, gbx, w["boxes"], step, w["dt"])
        step += 1
    npairs = int(sums[12])
    l0 = ctx.dmb_launch_count()
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        ctx.dmb_step_batched(dm, dbx, gas, gbx, w["boxes"], step, w["dt"], want_sums=False)
        step += 1
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    nd, ng = len(w["dm"]["h"]), len(w["gas"]["h"])
    names = ["grid", "search", "meanfield", "mc", "kick"]
    line = {"metric": "pair_interactions_per_s", "value": npairs * a.steps / (ms * 1e-3), "unit": "pairs/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 pairs, f64 sums",
            "data": "synthetic",
            "config": {"workload": f"boxes64: 64 periodic boxes, {nd} DM + {ng} gas in total, per-box sigma0, "
                                   f"m_chi, T and counts log-uniform", "pairs_per_step": npairs,
                       "parallelism": "replicas x1"},
            "particles_stepped_per_s": (nd + ng) * a.steps / (ms * 1e-3),
            "graph": True, "graph_launches_per_step": 1,
            "kernels_per_step": int(ctx.dmb_launch_count() - l0) // max(a.steps, 1),
            "direct_ms_per_step": direct_ms,
            "stage_ms_direct": {n: float(v) / max(nsteps, 1) for n, v in zip(names, stage_ms[:5])},
            "gpu_launches": int(ctx.dmb_launch_count() - l0), "clocks": clk, "peak_kind": peak_kind}
    print(json.dumps(line))
    ctx.close()
    return 0


def run_boxtest(a, peaks, peak_kind):
    """The App. F periodic-box test (fiducial row of Table test_params, 32^3 + 32^3 particles):
    `steps` steps of the interaction step plus the drift, after `warmup` steps; the run's own
    snapshots are not taken inside the timed steps."""
    import torch
    from paper_2603_24688_gb300 import boxtest as BT
    BT.run("fiducial", t_end=a.warmup * 1e-3, dt=1e-3, snap=10 ** 9)
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    r = BT.run("fiducial", t_end=a.steps * 1e-3, dt=1e-3, snap=10 ** 9)
    clk = clocks.stop()
    ms = r["ms_per_step"]
    row = r["row"]
    n_part = row["N_chi"] + row["N_B"]
    line = {"metric": "pair_interactions_per_s", "value": r["n_pairs"] / (ms * 1e-3), "unit": "pairs/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 pairs, f64 sums", "data": "synthetic",
            "config": {"workload": "boxtest: App. F fiducial periodic box, 32^3 DM + 32^3 gas, m_chi = 2 m_p, "
                                   "sigma = 1e-26 cm^2, V_chi = 200 km/s, T_chi = 1e6 K, T_B = 1e4 K, dt = 1e-3, "
                                   "dmb_step + drift per step", "pairs_per_step": r["n_pairs"],
                       "parallelism": "replicas x1"},
            "particles_stepped_per_s": n_part / (ms * 1e-3), "scatters": r["scatters"],
            "clocks": clk, "peak_kind": peak_kind}
    print(json.dumps(line))
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload in ("galaxy40M", "boxes64", "boxtest"):
        import torch
        from paper_2603_24688_gb300 import build
        build.build()
        peaks, peak_kind = load_peaks()
        fn = {"galaxy40M": run_substeps, "boxes64": run_boxes, "boxtest": run_boxtest}[a.workload]
        return fn(a, peaks, peak_kind)
    import torch
    from paper_2603_24688_gb300 import build, dmb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    peaks, peak_kind = load_peaks()

    w = make_workload(a.workload, a.n, seed_offset=rank)
    dm = dmb.to_device(w["dm"])
    gas = dmb.to_device(w["gas"])
    stream = torch.cuda.current_stream()
    modes = {"closed": dmb.DMB_RATE_CLOSED, "quad": dmb.DMB_RATE_QUAD, "mlp": dmb.DMB_RATE_MLP}
    prm = w["params"]

    def new_ctx(rate):
        c = dmb.Context(prm["sigma0_cm2"], prm["n"], prm["m_chi_mp"], prm["v0_kms"], prm["periodic"],
                        tuple(prm["box"]), prm["seed"], fp64=a.fp64, rate_mode=modes[rate], stream=stream)
        c.dmb_set_surrogate_epilogue(a.surrogate_epilogue)
        c.dmb_set_pair_weights(a.pair_weights)
        return c

    surrogate = None
    train_report = None
    if a.rate == "mlp" or not a.no_compare:
        tctx = new_ctx("mlp")
        train_report = tctx.dmb_train_surrogate(**(dict(nsamples=1 << 18, epochs=2, seed=11) if a.quick_train
                                                    else TRAIN))
        surrogate = tctx.dmb_surrogate_params()
        tctx.close()
    ctx = new_ctx(a.rate)
    if a.rate == "mlp":
        ctx.dmb_load_surrogate(surrogate)
    shapes, tune_times = (None, None)
    shapes_from = None
    if not a.no_autotune:
        # the autotuner's choice persists per workload (host JSON written by the library)
        cache = os.path.join(ROOT, "paper_2603_24688_gb300", "_build", "tuned_shapes.json")
        key = f"{a.workload}.n{a.n}.{a.rate}" + (".fp64" if a.fp64 else "")
        if not a.retune and ctx.dmb_load_shapes(cache, key):
            shapes, shapes_from = ctx.dmb_get_shapes(), "loaded from " + os.path.relpath(cache, ROOT)
        else:
            shapes, tune_times = ctx.dmb_autotune(dm, gas)   # reads the state only
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            ctx.dmb_save_shapes(cache, key)
            shapes_from = "dmb_autotune on this state"
    dt = w["dt"]
    step = 0
    sums = None
    for _ in range(a.warmup):
        sums = ctx.dmb_step(dm, gas, step, dt)
        step += 1
    torch.cuda.synchronize()
    npairs = int(sums[12]) if sums is not None else 0

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region --------------------------------------------------
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) if rank == 0 else None
    ctx.dmb_set_timing(True)
    launches0 = ctx.dmb_launch_count()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pairs_total = 0
    for _ in range(a.steps):
        sums = ctx.dmb_step(dm, gas, step, dt)
        pairs_total += int(sums[12])
        step += 1
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = ctx.dmb_launch_count() - launches0
    stage_ms, nsteps = ctx.dmb_stage_times()
    ctx.dmb_set_timing(False)
    clk = clocks.stop() if clocks else None
    ms_max, pairs_all = reduce_across_ranks(ms, pairs_total, dist)
    value = pairs_all / (ms_max * 1e-3)
    nparticles = len(w["dm"]["h"]) + len(w["gas"]["h"])

    # ---- roofline of the dominant kernel ----------------------------------------------
    names = ["grid", "search", "meanfield", "mc", "kick"]
    per_step = stage_ms[:5] / max(nsteps, 1)
    surrogate_ms = float(stage_ms[5] / max(nsteps, 1))
    dom = int(np.argmax(per_step))
    kern = {"grid": "k_radix_scatter+k_gather+k_morton", "search": "k_pair_search",
            "meanfield": "k_meanfield", "mc": "k_mc", "kick": "k_kick_gas"}[names[dom]]
    roof = None
    fmax_ghz = peaks.get("sm_max_mhz", 2070.0) / 1e3
    # whether the step's own search stored pair weights (then the geometry is the search's work)
    w_used = a.pair_weights == 1 and not a.fp64
    alu_peak = SMS * LANES * fmax_ghz * 1e9 / 1e12          # T lane-ops/s

    def roofline(stage):
        k = names.index(stage)
        t = per_step[k] * 1e-3
        if stage == "meanfield" and a.rate == "mlp" and surrogate_ms > 0:
            # the surrogate's tensor-core pass (k_mlp_tc), timed alone inside the step: bound by
            # the tensor cores (bf16 operands, float32 accumulation)
            ts = surrogate_ms * 1e-3
            tpeak = peaks.get("bf16_tflops_sustained", 1700.0)
            ach = MLP_FLOP_PER_PAIR * npairs / ts / 1e12
            issued = MLP_TENSOR_FLOP_PER_PAIR * npairs / ts / 1e12
            epi = a.surrogate_epilogue == 1
            per_pair = MLP_MF_DRAM_BYTES_PER_PAIR if epi else MLP_DRAM_BYTES_PER_PAIR
            traffic = None if per_pair is None else per_pair * npairs
            return {"bound": "tensor", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s", "frac": ach / tpeak,
                    "traffic": traffic, "traffic_unit": "bytes per launch",
                    "traffic_source": "ncu capture of this kernel on galaxy1M, scaled by the pair count",
                    "algorithmic_bytes": (MLP_MF_ALGO_BYTES_PER_PAIR if epi else MLP_ALGO_BYTES_PER_PAIR) * npairs,
                    "kernel": ("k_mlp_tc (surrogate 4 -> 128 -> 128 -> 128 -> 2 per pair, with the gas mean field "
                               "summed in its epilogue; the time includes the float64 finish per gas row)") if epi
                    else "k_mlp_tc (surrogate pass: 4 -> 128 -> 128 -> 128 -> 2 per pair, rates stored)",
                    "flop_per_pair": MLP_FLOP_PER_PAIR,
                    "issued_tflops": issued, "issued_flop_per_pair": MLP_TENSOR_FLOP_PER_PAIR,
                    "peak_source": f"bf16_tflops_sustained of MEASURED_PEAKS.json ({peak_kind})",
                    "kernel_ms": surrogate_ms}
        if stage in OPS_PER_PAIR:
            table = OPS_PER_PAIR_F32 if w_used else OPS_PER_PAIR
            ops = table[stage] if not (stage == "meanfield" and a.rate == "quad") else \
                QUAD_OPS_PER_PAIR - (GEOM_OPS_PER_PAIR if w_used else 0.0)
            kern = {"meanfield": "k_meanfield", "mc": "k_mc"}[stage]
            ach = ops * npairs / t / 1e12
            return {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "Tops/s", "frac": ach / alu_peak,
                    "traffic": None, "kernel": kern, "ops_per_pair": ops,
                    "peak_source": "152 SMs x 128 FP32/INT lanes x max SM clock (unit counts)"}
        return None

    order = np.argsort(-per_step)
    for k in order:                      # the slowest stage that has a per-pair roofline
        roof = roofline(names[k])
        if roof is not None:
            roof["stage_share"] = float(per_step[k] / per_step.sum())    # the stage's share of the step
            if "kernel_ms" in roof:                                         # the kernel's own share
                roof["kernel_share"] = float(roof["kernel_ms"] / per_step.sum())
            break
    stages = {n: float(v) for n, v in zip(names, per_step)}
    if a.fp64:
        for n in ("meanfield", "mc"):
            r = roofline(n)
            stages[n + "_frac"] = r["frac"] if r else None
    else:
        # the mean-field kernel alone (the surrogate pass before it is the tensor roofline) and the
        # Monte Carlo, each against the lane-operation roofline
        table = OPS_PER_PAIR_F32 if w_used else OPS_PER_PAIR
        mf_ops = {"closed": table["meanfield"], "quad": QUAD_OPS_PER_PAIR - (GEOM_OPS_PER_PAIR if w_used else 0.0),
                  "mlp": table["meanfield"] - RATE_OPS_CLOSED}[a.rate]
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        if a.rate == "mlp" and a.surrogate_epilogue == 1:
            # the mean field runs inside the surrogate's kernel: no kernel of its own to time
            stages["meanfield_kernel_ms"] = None
            stages["meanfield_frac"] = None
            stages["meanfield_in"] = "k_mlp_tc epilogue"
        else:
            t_mf = (per_step[2] - surrogate_ms) * 1e-3
            stages["meanfield_kernel_ms"] = float(per_step[2] - surrogate_ms)
            stages["meanfield_frac"] = mf_ops * npairs / t_mf / 1e12 / alu_peak
            if w_used:   # with the stored weights the kernel streams its pairs: its memory roofline
                stages["meanfield_hbm_frac"] = MF_BYTES_PER_PAIR[a.rate] * npairs / t_mf / 1e9 / hbm_peak
        stages["mc_frac"] = table["mc"] * npairs / (per_step[3] * 1e-3) / 1e12 / alu_peak
        stages["pair_weights"] = bool(w_used)
    # the pair search: candidate distance tests of the count pass (after the ballot prefilter) at
    # SEARCH_OPS_PER_TEST lane operations each, and (float32) the pair geometry of every pair in the
    # emit pass, over the whole search stage's time
    st = ctx.dmb_search_stats()
    tests = float(st[0][2])
    search_ops = tests * SEARCH_OPS_PER_TEST + (GEOM_OPS_PER_PAIR * npairs if w_used else 0.0)
    stages["search_candidate_tests"] = tests
    stages["search_frac"] = search_ops / (per_step[1] * 1e-3) / 1e12 / alu_peak if per_step[1] > 0 else None

    # ---- the other rate providers: mean-field stage time on the same state ------------------
    providers = {a.rate: {"meanfield_ms": float(per_step[2])}}
    if not a.no_compare:
        for rate in ("closed", "quad", "mlp"):
            if rate == a.rate:
                continue
            c2 = new_ctx(rate)
            if rate == "mlp":
                c2.dmb_load_surrogate(surrogate)
            if shapes is not None:
                c2.dmb_set_shapes(shapes)
            c2.dmb_set_timing(True)
            dm2 = {k: v.clone() for k, v in dm.items()}
            gas2 = {k: v.clone() for k, v in gas.items()}
            for _ in range(2):
                c2.dmb_step(dm2, gas2, step, dt)
            ms2, n2 = c2.dmb_stage_times()
            providers[rate] = {"meanfield_ms": float(ms2[2] / max(n2, 1))}
            c2.close()
            del dm2, gas2
        if "quad" in providers and "mlp" in providers:
            providers["mlp_speedup_over_quad"] = providers["quad"]["meanfield_ms"] / providers["mlp"]["meanfield_ms"]
        # the cross-section scan of the workload: every rate provider's mean field and the whole
        # surrogate step at each n, with the surrogate's rate error at that n
        per_n = {}
        pair_inputs = None
        for n in SCAN_N:
            row = {}
            for rate in ("closed", "quad", "mlp"):
                c2 = dmb.Context(prm["sigma0_cm2"], n, prm["m_chi_mp"], prm["v0_kms"], prm["periodic"],
                                 tuple(prm["box"]), prm["seed"], fp64=a.fp64, rate_mode=modes[rate], stream=stream)
                c2.dmb_set_surrogate_epilogue(a.surrogate_epilogue)
                c2.dmb_set_pair_weights(a.pair_weights)
                if rate == "mlp":
                    c2.dmb_load_surrogate(surrogate)
                if shapes is not None:
                    c2.dmb_set_shapes(shapes)
                c2.dmb_set_timing(True)
                dm2 = {k: v.clone() for k, v in dm.items()}
                gas2 = {k: v.clone() for k, v in gas.items()}
                for _ in range(2):
                    c2.dmb_step(dm2, gas2, step, dt)
                ms2, n2 = c2.dmb_stage_times()
                row[rate + "_meanfield_ms"] = float(ms2[2] / max(n2, 1))
                if rate == "mlp":
                    row["mlp_step_ms"] = float(ms2[:5].sum() / max(n2, 1))
                    row["surrogate_fallback_pairs"] = int(c2.dmb_surrogate_fallbacks())
                c2.close()
                del dm2, gas2
            row["mlp_speedup_over_quad"] = row["quad_meanfield_ms"] / row["mlp_meanfield_ms"]
            if surrogate is not None:
                row["surrogate_rate_error"] = surrogate_errors(surrogate, n, prm)
                # the same over the (s, tau, m_chi) this workload's pairs can reach, and at the
                # inputs of 2^20 of its pairs drawn at random (those inside the training box; the
                # others take the quadrature)
                row["surrogate_rate_error_workload"] = surrogate_errors(surrogate, n, prm, tau=workload_tau(w),
                                                                        m_chi=prm["m_chi_mp"])
                if pair_inputs is None:
                    c3 = new_ctx("closed")
                    pair_inputs = workload_pair_inputs(c3, dm, gas, prm)
                    c3.close()
                ps, pt = pair_inputs
                inb = (ps >= 1e-2) & (ps <= 1e2) & (pt >= 1e-3) & (pt <= 1e2)
                pe = rate_errors(surrogate, n, prm, ps[inb], pt[inb], np.full(int(inb.sum()), prm["m_chi_mp"]))
                pe.update(sampled=int(ps.size), in_box=int(inb.sum()))
                row["surrogate_rate_error_pairs"] = pe
            per_n[str(n)] = row
        providers["per_n"] = per_n
    if train_report is not None:
        providers["surrogate_training"] = {"seconds": float(train_report[5]), "steps": int(train_report[6]),
                                           "samples": int(train_report[7]),
                                           "val_mean_rel_err_A": float(train_report[3]),
                                           "val_mean_rel_err_B": float(train_report[4]),
                                           "val_max_rel_err_A": float(train_report[1]),
                                           "val_max_rel_err_B": float(train_report[2])}

    # ---- end to end through the C ABI with host buffers ---------------------------------
    # Every step copies its inputs from pinned host memory and its resulting state back, inside
    # the timed region, pipelined over two device buffer sets: step k+1's inputs travel on a copy
    # stream while step k runs, and step k's results come back while step k+1 runs.
    e2e = None
    if a.e2e_steps > 0:
        # the pinned host buffers on the GPU's own NUMA node (first touch by a thread bound to its
        # CPUs), so that the copies do not cross between host sockets
        cpus_before = os.sched_getaffinity(0)
        numa_node = bind_to_gpu_numa_node(torch.cuda.current_device())
        host = {}
        for sp, src in (("dm", dm), ("gas", gas)):
            host[sp] = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in src.items()}
            for k, v in src.items():
                host[sp][k].copy_(v)
        outs = [{"dm_vel": torch.empty_like(dm["vel"], device="cpu").pin_memory(),
                 "gas_vel": torch.empty_like(gas["vel"], device="cpu").pin_memory(),
                 "gas_T": torch.empty_like(gas["T"], device="cpu").pin_memory()} for _ in range(2)]
        h2d = sum(v.numel() * v.element_size() for sp in host.values() for v in sp.values())
        d2h = sum(v.numel() * v.element_size() for v in outs[0].values())
        bufs = [(dm, gas), ({k: v.clone() for k, v in dm.items()}, {k: v.clone() for k, v in gas.items()})]
        cstream = torch.cuda.Stream()
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        done = [None, None]
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        cstream.wait_stream(stream)

        def h2d_into(k):
            d_, g_ = bufs[k % 2]
            with torch.cuda.stream(cstream):
                if done[k % 2] is not None:
                    cstream.wait_event(done[k % 2])          # the set's previous step is finished
                for sp, dst in (("dm", d_), ("gas", g_)):
                    for name, v in dst.items():
                        v.copy_(host[sp][name], non_blocking=True)
                ready[k % 2].record(cstream)

        h2d_into(0)
        for k in range(a.e2e_steps):
            if k + 1 < a.e2e_steps:
                h2d_into(k + 1)                               # behind step k
            d_, g_ = bufs[k % 2]
            stream.wait_event(ready[k % 2])
            ctx.dmb_step(d_, g_, step, dt, want_sums=False)
            step += 1
            ev = torch.cuda.Event()
            ev.record(stream)
            done[k % 2] = ev
            o = outs[k % 2]
            with torch.cuda.stream(cstream):
                cstream.wait_event(ev)
                o["dm_vel"].copy_(d_["vel"], non_blocking=True)
                o["gas_vel"].copy_(g_["vel"], non_blocking=True)
                o["gas_T"].copy_(g_["T"], non_blocking=True)
        stream.wait_stream(cstream)
        f1.record(stream)
        barrier()
        ms_e, pairs_e = reduce_across_ranks(f0.elapsed_time(f1), npairs * a.e2e_steps, dist)
        # the copies alone (no step running beside them), for the record
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c2 = torch.cuda.Event(enable_timing=True)
        d_, g_ = bufs[0]
        c0.record(stream)
        for sp, dst in (("dm", d_), ("gas", g_)):
            for name, v in dst.items():
                v.copy_(host[sp][name], non_blocking=True)
        c1.record(stream)
        outs[0]["dm_vel"].copy_(d_["vel"], non_blocking=True)
        outs[0]["gas_vel"].copy_(g_["vel"], non_blocking=True)
        outs[0]["gas_T"].copy_(g_["T"], non_blocking=True)
        c2.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": pairs_e / (ms_e * 1e-3), "unit": "pairs/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "pipelined": "inputs of step k+1 copied while step k runs; results of step k copied while step k+1 runs",
               "ms_per_step": ms_e / a.e2e_steps,
               "h2d_ms_alone": c0.elapsed_time(c1), "d2h_ms_alone": c1.elapsed_time(c2),
               "host_numa_node": numa_node}
        os.sched_setaffinity(0, cpus_before)      # the CPU baseline below uses every host core

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        rate1, n1, t1, desc1 = cpu_oracle_sample(w)
        rate, n_s, t_s, cores, desc = cpu_oracle_all_cores(w)
        cpu = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": desc,
               "host_cpus": host_cpu_count(),
               "single_thread": {"value": rate1, "unit": "pairs/s", "cores": 1, "sample": desc1}}

    if rank == 0:
        line = {"metric": "pair_interactions_per_s", "value": value, "unit": "pairs/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.fp64 else "f32 pairs, f64 sums",
                "data": "synthetic",
                "config": {"workload": workload_desc(a, w),
                           "rate_provider": {"mlp": "learned surrogate (tcgen05 tensor cores)",
                                             "quad": "64-point Gauss-Legendre quadrature",
                                             "closed": "closed-form 1F1"}[a.rate],
                           "pairs_per_step": npairs,
                           "l2": "inputs (~1 GB) larger than L2; no flush", "parallelism": f"replicas x{world}"},
                "particles_stepped_per_s": nparticles * world / (ms_max * 1e-3 / a.steps),
                "stage_ms": dict(stages, surrogate_pass=surrogate_ms), "rate_providers": providers,
                "launch_shapes": shapes, "launch_shapes_from": shapes_from, "gpu_launches": int(launches), "roofline": roof,
                "peak_kind": peak_kind,
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
