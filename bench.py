#!/usr/bin/env python
"""Benchmark of the CKKS hybrid key-switching path on one GB300 (or N replicas).

Workload (single-op path): logN=16 (N=65536), 30 ciphertext limbs of 54-bit
primes, K=10 special 60-bit primes, dnum=3 (10 limbs per digit).  One step is
  HMult+relin of a ciphertext pair  ->  Rescale of the product (30 -> 29 limbs)
  HRotate of a ciphertext by 2^(k mod 15) slots (15 rotation keys)
with every input resident in HBM.  The metric counts HMult+relin and HRotate
operations (two per step); the Rescale time is inside the timed region.

Inputs are seeded synthetic residues (uniform mod each prime, from the shared
generator in seeded_inputs.py); keys are uniform residues of the key shape
(computationally indistinguishable from real RLWE keys, and the kernels'
work does not depend on their values).  A pool of 8 ciphertext pairs and the
16 keys (1.9 GiB) are cycled, so each step touches >400 MB: more than the
129 MB L2 between repeats.

Modes
  python bench.py [--gpus N --steps K --warmup W]      the CUDA library
  python bench.py --impl reference ...                 the CPU oracle (reference arm)
Multi-GPU runs are replicas (one independent workload per rank, no collective
on the data path; torch.distributed only for the barrier and the max-time).
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

import seeded_inputs as si  # noqa: E402

METRIC = "HMult+relin & HRotate ops/s (logN=16,L=30,dnum=3)"
POOL = 8
N_ROT = 15


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fides", choices=["fides", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=8.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 128-ciphertext batched workload")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default NTT tile widths")
    ap.add_argument("--batch-ops", type=int, default=128)
    ap.add_argument("--no-serving", action="store_true", help="skip the request-server workload")
    ap.add_argument("--no-ops", action="store_true", help="skip hoisted rotations, linear transform, element-wise")
    ap.add_argument("--no-bootstrap", action="store_true", help="skip the bootstrapping workload")
    ap.add_argument("--clocks-dir", default=None, help="where the sampled nvidia-smi clock log is written")
    ap.add_argument("--bootstrap-only", action="store_true",
                    help="run only the bootstrapping workload and print its JSON (for profiler launch lists)")
    ap.add_argument("--bootstrap-batch", type=int, default=8)
    ap.add_argument("--bootstrap-lanes", type=int, default=2,
                    help="programs (each with its own work buffer) run on this many streams of one context")
    ap.add_argument("--ops-only", action="store_true",
                    help="run only the hoisted-rotation / linear-transform / element-wise legs (profiler captures)")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-lanes", type=int, default=2)
    ap.add_argument("--serve-max-batch", type=int, default=32)
    ap.add_argument("--serve-saturate", type=int, default=6000, help="requests of the closed-loop run")
    ap.add_argument("--serve-depth", type=int, default=256, help="outstanding requests of the closed-loop run")
    ap.add_argument("--small", action="store_true",
                    help="one ciphertext pair and two keys (for profiler captures; not a bench line)")
    args = ap.parse_args()
    if args.small:
        global POOL, N_ROT
        POOL, N_ROT = 1, 1
    return args


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "fides" else "gloo"
        if args.impl == "fides":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, directory: str | None = None):
        import tempfile
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(directory or tempfile.gettempdir(), "clocks_rank%d.csv" % gpu_index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
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
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload_config(P, world):
    """The `config` object of the JSON line (the same for both arms)."""
    return {"workload": "single-op path logN=16 L=30 K=10 dnum=3: HMult+relin, Rescale, HRotate(2^(k mod 15))",
            "logN": P.logN, "limbs": P.nq, "special_primes": P.nk, "dnum": P.dnum, "q_bits": P.q_bits,
            "p_bits": P.p_bits, "ops_per_step": 2,
            "l2": "inputs larger than L2: 8 ciphertext pairs + 16 keys (1.9 GiB) cycled, >400 MB per step",
            "parallelism": "replicas" if world > 1 else "single"}


def workload_inputs(P, q, p, seed):
    """Host arrays of the workload: POOL ciphertext pairs and 16 keys."""
    st = si.Stream(seed, 10)
    N = 1 << P.logN
    A = [np.stack([si.uniform_poly(st, q, N) for _ in range(2)]) for _ in range(POOL)]
    B = [np.stack([si.uniform_poly(st, q, N) for _ in range(2)]) for _ in range(POOL)]
    keys = [np.stack([np.stack([si.uniform_poly(st, q + p, N) for _ in range(2)]) for _ in range(P.dnum)])
            for _ in range(1 + N_ROT)]
    return A, B, keys


def launch_model(nl, K, alpha, N, bconv="k_bconv_tc"):
    """Per-step launches of the library's kernels with their algorithmic work.

    Unit of an NTT pass: one limb (N u64 read + N written = 16 N bytes,
    (N/2)*log2(N)/2 butterflies = one Shoup product each).  Element-wise
    kernels count the limbs they must read and write once.  Returns a list of
    (kernel, bytes, modmuls)."""
    W = 8 * N
    half_bfly = (N // 2) * 8          # butterflies of one pass (8 of the 16 stages) per limb
    beta = -(-nl // alpha)
    ne = nl + K
    L = []

    def ntt(direction, limbs, extra_bytes=0, extra_mm=0, ninv=False, first_bytes=0, first_mm=0):
        # two passes; the first carries any fused prologue, the second any fused epilogue
        L.append(("k_ntt_%s_%s" % (direction, "rows" if direction == "inv" else "cols"),
                  2 * W * limbs + first_bytes, half_bfly * limbs + first_mm))
        L.append(("k_ntt_%s_%s" % (direction, "cols" if direction == "inv" else "rows"),
                  2 * W * limbs + extra_bytes, half_bfly * limbs + extra_mm + (N * limbs if ninv else 0)))

    def keyswitch(mode0, mode1, prep):
        # HMult: the tensor product as its own pass (reads a, b, writes d0,
        # d1, d2 with 4 products), then a plain ModUp INTT of d2.  HRotate:
        # the INTT's first pass gathers c0, c1 and writes sigma(c0), sigma(c1)
        if prep == "tensor":
            L.append(("k_tensor", 7 * W * nl, 4 * N * nl))
            fb, fm = 0, 0
        else:
            fb, fm = 3 * W * nl, 0
        ntt("inv", nl, ninv=True, first_bytes=fb, first_mm=fm)
        ntgt = beta * ne - nl
        L.append((bconv, W * (nl + ntgt), N * sum(min(alpha, nl - j * alpha) * (ne - min(alpha, nl - j * alpha)) for j in range(beta))))
        ntt("fwd", ntgt)
        L.append(("k_inner", W * (beta * ne + 2 * beta * ne + 2 * ne), N * 2 * beta * ne))
        ntt("inv", 2 * K, ninv=True)                                 # ModDown: P-limbs to coefficients
        L.append((bconv, W * (2 * K + 2 * nl), N * 2 * K * nl))
        extra = W * nl * (2 + mode0 + mode1)                         # aux reads (+ out reads when accumulating)
        ntt("fwd", 2 * nl, extra_bytes=extra, extra_mm=2 * N * nl)

    # HMult+relin
    keyswitch(1, 1, "tensor")
    # Rescale of the product
    ntt("inv", 2, ninv=True)
    ntt("fwd", 2 * (nl - 1), extra_bytes=W * 2 * (nl - 1), extra_mm=N * 4 * (nl - 1))
    # HRotate
    keyswitch(1, 0, "permute")
    return L


def op_work(nl, K, alpha, N):
    """Compulsory HBM bytes and modmul-equivalents of one HMult+relin, HRotate
    and Rescale at nl limbs: inputs + the key limbs in use + outputs; (beta+2)
    (nl+K) transforms of (N/2) log2 N butterflies, the conversions' multiply-adds
    and the element-wise products (the tensor product for HMult)."""
    import math
    W = 8 * N
    beta, ne = -(-nl // alpha), nl + K
    digits = [min(alpha, nl - j * alpha) for j in range(beta)]
    bfly = (N // 2) * int(math.log2(N))
    ks_mm = (beta + 2) * ne * bfly + N * (sum(a * (ne - a) for a in digits) + 2 * K * nl) \
        + N * (sum(digits) + 2 * beta * ne + 2 * K + 2 * nl)
    return {"hmult": (W * (4 * nl + 2 * beta * ne + 2 * nl), ks_mm + N * 4 * nl),
            "rotate": (W * (2 * nl + 2 * beta * ne + 2 * nl), ks_mm),
            "rescale": (W * (2 * nl + 2 * (nl - 1)), (2 + 2 * (nl - 1)) * bfly + N * 2 * (nl - 1))}


def bconv_tc_flops(nl, K, alpha, N):
    """fp16 flops one step's tensor-core conversions issue: per job of ns
    sources and nd targets, 2 * N coefficients * 8 nd output columns * 8 nsp
    byte rows, nsp = ns + 1 (the offset column) rounded up to even.  Two key
    switches, each one ModUp job per digit and two ModDown jobs."""
    beta, ne = -(-nl // alpha), nl + K
    per_ks = 0
    for j in range(beta):
        ns = min(alpha, nl - j * alpha)
        per_ks += 2 * N * 8 * (ne - ns) * 8 * ((ns + 2) & ~1)
    per_ks += 2 * (2 * N * 8 * nl * 8 * ((K + 3) & ~1))   # ModDown images carry the correction column
    return 2 * per_ks


def tensor_peak():
    """Measured dense bf16 TFLOP/s (burst) from MEASURED_PEAKS.json, or None."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        mp = json.load(open(path))
        return float(mp["hbm_gbs"]), "measured", float(mp.get("sm_max_mhz", 2070.0))
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback", 2070.0


# ALU roofline of a 64-bit Shoup product, from unit counts and the SM clock:
# 152 SMs x 64 lanes of the integer multiply (fmaheavy) pipe per clock, and 16
# lane-cycles per product -- its 10 IMAD-class instructions (4 for the high
# half of a 64x64 product, 3 for each low half) hold a sub-partition's pipe 32
# cycles per warp of 32 products (ncu on the register-resident microbenchmark:
# 10.0 FMA-pipe warp instructions and 1.00 pipe cycle per product per
# sub-partition, the pipe 95.6 % busy).
LANE_CYCLES_PER_MODMUL = 16
FMAHEAVY_LANES_PER_CLK_SM = 64
SMS = 152

# What limits each kernel, from its ncu profile: the NTT passes the integer
# multiply pipe, the inner and tensor products DRAM, the conversion the
# tensor-core issue path.
KERNEL_BOUND = {"k_ntt": "alu", "k_inner": "hbm", "k_tensor": "hbm", "k_elem": "hbm", "k_ptmac": "hbm",
                "k_bconv_tc": "tensor"}


def kernel_bound(name):
    return next((v for k, v in KERNEL_BOUND.items() if name.startswith(k)), None)


def run_fides(args, world, rank, local):
    import torch

    import paper_2507_04775_gb300 as fides

    torch.cuda.set_device(local)
    P = si.FULL
    q = fides.find_primes(P.logN, P.q_bits, P.nq)
    p = fides.find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    ctx = fides.Context(P.logN, q, p, P.dnum)
    t_tune = time.perf_counter()
    if not args.no_autotune:
        ctx.autotune(128)
    t_tune = time.perf_counter() - t_tune
    tiles = {name: {n: "%d/%d" % (ctx.ntt_tile(k, n) >> 8, ctx.ntt_tile(k, n) & 255) for n in (2, 20, 30, 58, 60, 90, 128)}
             for k, name in enumerate(("fwd_cols", "fwd_rows", "inv_rows", "inv_cols"))}
    N, nl = ctx.N, P.nq
    A, B, keys = workload_inputs(P, q, p, si.workload_seed(1) + 1000 * rank)
    dA = [fides.to_device(x) for x in A]
    dB = [fides.to_device(x) for x in B]
    dK = [fides.to_device(x) for x in keys]
    # switching keys as registered handles: the relinearisation key and the
    # keys of the rotations by 2^k (uniform residues; see the module docstring)
    rlk = ctx.relin_key(dK[0])
    rks = [ctx.rotation_key(dK[1 + k], 1 << k) for k in range(N_ROT)]
    out_m = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
    out_r = torch.empty_like(out_m)
    out_s = torch.empty(2 * (nl - 1) * N, dtype=torch.int64, device="cuda")
    scale = 2.0 ** P.log_scale

    def step(k, a=None, b=None):
        i = k % POOL
        a = dA[i] if a is None else a
        b = dB[i] if b is None else b
        s = ctx.hmult(a, b, nl, rlk, out_m, scale, scale)
        ctx.rescale(out_m, nl, out_s, s)
        ctx.rotate(a, nl, 1 << (k % N_ROT), rks[k % N_ROT], out_r, scale)

    clocks = Clocks(local, args.clocks_dir)
    clocks.start()             # sampling runs through the warm-up and the timed region
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    # ---------------- timed region (inputs resident in HBM) ----------------
    launches0 = fides.kernel_launches()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = fides.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world)
    ops = 2 * args.steps * world
    value = ops / (ms_max / 1e3)

    # ------- the same steps with HMult and Rescale as one call (reported
    # beside the single-op value, which stays the headline) -------
    def step_fused(k):
        i = k % POOL
        ctx.hmult_rescale(dA[i], dB[i], nl, rlk, out_s, scale, scale)
        ctx.rotate(dA[i], nl, 1 << (k % N_ROT), rks[k % N_ROT], out_r, scale)

    for k in range(args.warmup):
        step_fused(k)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step_fused(k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fused = max_over_ranks(e0.elapsed_time(e1), world)
    fused = {"workload": "the same steps with fides_hmult_rescale (HMult+relin and Rescale in one key switch, "
                         "residues equal to the two calls), then HRotate",
             "value": round(ops / (ms_fused / 1e3), 2), "unit": "ops/s", "ms_per_step": round(ms_fused / args.steps, 4)}

    # ------- the same steps under round-to-nearest ModDown and Rescale (the
    # mode whose decryption error meets 2^-20 at this size) -------
    ctx.set_rounding(True)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.set_rounding(False)
    ms_near = max_over_ranks(e0.elapsed_time(e1), world)
    nearest = {"workload": "the same steps with the context in round-to-nearest mode (centred ModDown conversion, "
                           "centred Rescale lift)",
               "value": round(ops / (ms_near / 1e3), 2), "unit": "ops/s", "ms_per_step": round(ms_near / args.steps, 4)}

    # ------- the same steps with HMult+Rescale on one registered stream and
    # HRotate on another (fides_ctx_add_stream gives each its own scratch):
    # the two chains' launches overlap and fill each other's dependent-launch
    # gaps (reported beside the single-stream headline) -------
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ctx.add_stream(sa)
    ctx.add_stream(sb)

    def run_two(n):
        ev = torch.cuda.Event()
        ev.record(stream)
        sa.wait_event(ev)
        sb.wait_event(ev)
        for k in range(n):
            i = k % POOL
            s = ctx.hmult(dA[i], dB[i], nl, rlk, out_m, scale, scale, stream=sa)
            ctx.rescale(out_m, nl, out_s, s, stream=sa)
            ctx.rotate(dA[i], nl, 1 << (k % N_ROT), rks[k % N_ROT], out_r, scale, stream=sb)
        done_b = torch.cuda.Event()
        done_b.record(sb)
        sa.wait_event(done_b)
        done_a = torch.cuda.Event()
        done_a.record(sa)
        stream.wait_event(done_a)

    run_two(args.warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    run_two(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_two = max_over_ranks(e0.elapsed_time(e1), world)
    two_streams = {"workload": "the same steps with HMult+relin and Rescale on one stream and HRotate on another, "
                               "both registered with the context (fides_ctx_add_stream)",
                   "value": round(ops / (ms_two / 1e3), 2), "unit": "ops/s",
                   "ms_per_step": round(ms_two / args.steps, 4)}

    # ------- the same K steps again, every launch bracketed by events -------
    # (events between launches serialise programmatic dependent launch, so
    # this pass gives per-kernel durations, not the value above)
    fides.trace_reset()
    fides.trace_enable(True)
    for k in range(args.steps):
        step(k)
    torch.cuda.synchronize()
    fides.trace_enable(False)
    ck = clocks.stop()
    trace = fides.trace_read()
    fides.trace_reset()
    peak_mm = fides.measure_modmul_peak()

    # ---------------- roofline of the dominant kernel ----------------
    kern = {k: v for k, v in trace.items() if k.startswith("k_")}
    top = max(kern, key=lambda k: kern[k][1])
    model = launch_model(nl, P.nk, ctx.alpha, N, "k_bconv_tc" if ctx.tensor_bconv else "k_bconv")
    per_kernel = {}
    for name, by, mm in model:
        d = per_kernel.setdefault(name, [0, 0, 0])
        d[0] += 1
        d[1] += by
        d[2] += mm
    mismatch = {k: (per_kernel.get(k, [0])[0] * args.steps, kern[k][0]) for k in kern
                if per_kernel.get(k, [0])[0] * args.steps != kern[k][0]}
    n_launch, by_step, mm_step = per_kernel[top]
    avg_ms = kern[top][1] / kern[top][0]
    bytes_per_launch = by_step / n_launch
    mm_per_launch = mm_step / n_launch
    hbm_peak, hbm_src, sm_max = peaks()
    hbm_ach = bytes_per_launch / (avg_ms / 1e3) / 1e9
    clk = (ck or {}).get("sm_mhz") or sm_max
    derived_alu = SMS * FMAHEAVY_LANES_PER_CLK_SM * sm_max * 1e6 / LANE_CYCLES_PER_MODMUL / 1e9   # Gmodmul/s
    alu_peak = derived_alu
    alu_ach = mm_per_launch / (avg_ms / 1e3) / 1e9
    traffic = load_traffic(top, bytes_per_launch)
    hbm = {"bound": "hbm", "achieved": round(hbm_ach, 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(hbm_ach / hbm_peak, 4), "traffic": traffic, "peak_source": hbm_src}
    alu = {"bound": "alu", "achieved": round(alu_ach, 1), "peak": round(alu_peak, 1), "unit": "Gmodmul/s",
           "frac": round(alu_ach / alu_peak, 4),
           "peak_source": ("derived: 152 SMs x 64 fmaheavy lanes x %.0f MHz / 16 lane-cycles per Shoup product "
                           "(10 IMAD-class instructions, 32 pipe cycles per warp; ncu on the microbenchmark)" % sm_max),
           "measured_microbenchmark": {
               "peak": round(peak_mm, 1), "frac": round(alu_ach / peak_mm, 4),
               "source": "measured in-run: register-resident Shoup products on all SMs (fides_measure_modmul_peak)"}}
    # every kernel of the step against both peaks (same launch model, same live
    # durations); the tensor-core conversion against the tensor peak instead
    kernel_roofline = {}
    tc_peak = tensor_peak()
    for name, (cnt, by, mm) in per_kernel.items():
        if name not in kern:
            continue
        avg = kern[name][1] / kern[name][0]
        ent = {"bound": kernel_bound(name), "launches_per_step": cnt, "avg_launch_us": round(avg * 1e3, 2),
               "hbm_frac": round(by / cnt / (avg / 1e3) / 1e9 / hbm_peak, 4)}
        if name == "k_bconv_tc":
            fl = bconv_tc_flops(nl, P.nk, ctx.alpha, N)
            ent["tensor_tflops"] = round(fl / cnt / (avg / 1e3) / 1e12, 1)
            ent["tensor_frac"] = round(fl / cnt / (avg / 1e3) / 1e12 / tc_peak, 4) if tc_peak else None
        else:
            ent["alu_frac"] = round(mm / cnt / (avg / 1e3) / 1e9 / alu_peak, 4)
        kernel_roofline[name] = ent
    # whole operations: compulsory bytes and modmul-equivalents against the
    # same two peaks (per op from its traced time, the step from the untraced one)
    work = op_work(nl, P.nk, ctx.alpha, N)
    op_roofline = {}
    for name, (by, mm) in work.items():
        key = "op_" + name
        if key in trace:
            us = trace[key][1] / trace[key][0] * 1e3
            op_roofline[name] = {"us": round(us, 1), "compulsory_mb": round(by / 1e6, 1),
                                 "modmul_equiv_m": round(mm / 1e6, 1),
                                 "hbm_frac": round(by / (us / 1e6) / 1e9 / hbm_peak, 4),
                                 "alu_frac": round(mm / (us / 1e6) / 1e9 / alu_peak, 4)}
    st_by = sum(v[0] for v in work.values())
    st_mm = sum(v[1] for v in work.values())
    st_ms = ms_max / args.steps
    op_roofline["step"] = {"ms": round(st_ms, 4), "compulsory_mb": round(st_by / 1e6, 1),
                           "modmul_equiv_m": round(st_mm / 1e6, 1),
                           "hbm_frac": round(st_by / (st_ms / 1e3) / 1e9 / hbm_peak, 4),
                           "alu_frac": round(st_mm / (st_ms / 1e3) / 1e9 / alu_peak, 4)}
    bound = kernel_bound(top)
    if bound not in ("alu", "hbm"):
        bound = "hbm" if hbm["frac"] >= alu["frac"] else "alu"
    roof = dict(hbm if bound == "hbm" else alu)
    roof["kernel"] = top
    roof["avg_launch_us"] = round(avg_ms * 1e3, 2)
    roof["other_bound"] = alu if roof["bound"] == "hbm" else hbm
    roof["clock_mhz_median"] = clk

    # ---------------- end to end through host buffers ----------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, world, ctx, A, B, rlk, rks, nl, N, scale)

    # ---------------- batched workload (many ciphertexts, uneven levels) ----------------
    batched = None
    if not args.no_batched and not args.small:
        batched = run_batched(args, ctx, dA, dB, rlk, rks, P, scale)

    # ---------------- request server (continuous batching) ----------------
    serving = None
    if not args.no_serving and not args.small:
        serving = run_serving(args, ctx, dA, dK, P, scale)

    # ---------------- hoisted rotations, linear transform, element-wise ----------------
    ops_extra = None
    if not args.no_ops and not args.small:
        ops_extra = run_ops(args, ctx, dA, dB, dK, P, scale)

    # ---------------- bootstrapping ----------------
    boot = None
    if not args.no_bootstrap and not args.small:
        boot = run_bootstrap(args)

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "ops/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(P, world),
        "per_op_us": {k[3:]: round(v[1] / v[0] * 1e3, 1) for k, v in trace.items() if k.startswith("op_")},
        "kernels_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in sorted(kern.items(), key=lambda x: -x[1][1])},
        "roofline": roof,
        "kernel_roofline": kernel_roofline,
        "op_roofline": op_roofline,
        "op_roofline_note": ("compulsory bytes = input ciphertexts + the key limbs in use + outputs, against the "
                             "measured HBM peak; modmul-equivalents = (beta+2)(nl+K) transforms x (N/2) log2 N "
                             "butterflies + conversion multiply-adds + element-wise products, against the derived "
                             "Shoup-product peak (conversions run on the tensor cores, so alu_frac overstates the "
                             "integer pipes' share)"),
        "kernel_roofline_note": ("algorithmic bytes (launch model) / live launch time against the measured HBM peak; "
                                 "modular products (Shoup butterflies, inner-product and tensor-product multiply-adds) "
                                 "/ live launch time against the derived Shoup-product peak; k_bconv_tc: fp16 "
                                 "flops of the MMA shapes it issues against the measured dense bf16 peak (fp16 runs "
                                 "at the bf16 rate); bound: what the kernel's ncu profile shows limits it"),
        "gpu_launches": int(launches),
        "clocks": ck,
        "e2e": e2e,
        "fused_hmult_rescale": fused,
        "round_to_nearest": nearest,
        "two_streams": two_streams,
        "batched": batched,
        "serving": serving,
        "ops": ops_extra,
        "bootstrap": boot,
        "autotune": {"ran": not args.no_autotune, "seconds": round(t_tune, 2), "ntt_tile_by_limbs": tiles},
    }
    if mismatch:
        result["launch_model_mismatch"] = mismatch
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(P, q, p, A, B, keys, args.cpu_seconds)
    elif rank == 0:
        result["cpu_baseline"] = None
    return result


def run_batched(args, ctx, dA, dB, rlk, rks, P, scale):
    """128 ciphertext pairs at levels drawn uniformly from {4..30}; each pair
    does HMult+relin then one HRotate (by a seeded power of two) of the
    product.  The batch runs as one captured CUDA graph (one launch per key-
    switch step per stage for the whole batch) and, for comparison, as one
    library call per operation on the same buffers."""
    import torch

    import paper_2507_04775_gb300 as fides
    st = si.Stream(si.workload_seed(2), 1)
    n = args.batch_ops
    levels = [4 + st.below(27) for _ in range(n)]
    rots = [st.below(N_ROT) for _ in range(n)]
    N = ctx.N
    ops, plain = [], []
    for i, nl in enumerate(levels):
        src_a, src_b = dA[i % POOL].view(2, P.nq, N), dB[i % POOL].view(2, P.nq, N)
        a = src_a[:, :nl].contiguous().view(-1)
        b = src_b[:, :nl].contiguous().view(-1)
        m = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
        r = torch.empty_like(m)
        ops.append(fides.Op(fides.OP_HMULT, a, nl, m, b=b, key=rlk, stage=0, scale_a=scale, scale_b=scale))
        ops.append(fides.Op(fides.OP_ROTATE, m, nl, r, key=rks[rots[i]], steps=1 << rots[i], stage=1,
                            scale_a=scale * scale))
        plain.append((a, b, m, r, nl, rots[i]))
    batch = fides.Batch(ctx, ops)
    info0 = batch.info()            # one launch group per stage
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t_tune = time.perf_counter()
        batch.autotune(stream)      # launch-group size and tensor-product placement
        t_tune = time.perf_counter() - t_tune
        info = batch.info()
        # per-kernel times of one traced run (events serialise the launches)
        fides.trace_reset()
        fides.trace_enable(True)
        batch.run(stream)
        stream.synchronize()
        fides.trace_enable(False)
        tr = fides.trace_read()
        fides.trace_reset()
        batch.capture(stream)
        for _ in range(2):
            batch.run(stream)
        stream.synchronize()
        reps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            batch.run(stream)
        e1.record(stream)
        stream.synchronize()
        ms_batch = e0.elapsed_time(e1) / reps

        def plain_run():
            for a, b, m, r, nl, k in plain:
                ctx.hmult(a, b, nl, rlk, m, scale, scale, stream=stream)
                ctx.rotate(m, nl, 1 << k, rks[k], r, scale * scale, stream=stream)
        plain_run()
        stream.synchronize()
        e0.record(stream)
        for _ in range(2):
            plain_run()
        e1.record(stream)
        stream.synchronize()
        ms_plain = e0.elapsed_time(e1) / 2
    batch.close()
    nops = 2 * n
    limbs = sum(levels)
    return {"workload": "%d ciphertexts, levels uniform on {4..30} (mean %.1f limbs), HMult+relin then HRotate" % (n, limbs / n),
            "ops": nops, "value": round(nops / (ms_batch / 1e3), 1), "unit": "ops/s",
            "ms_per_batch": round(ms_batch, 3), "plain_value": round(nops / (ms_plain / 1e3), 1),
            "plain_ms": round(ms_plain, 3), "speedup": round(ms_plain / ms_batch, 3),
            "graph": True, "kernels_per_batch": info["launches"],
            "kernels_plain": n * 22, "scratch_gib": round(info["scratch_bytes"] / 2**30, 2),
            "autotune": {"seconds": round(t_tune, 1), "group_limbs": info["group_limbs"], "groups": info["groups"],
                         "tensor_split": info["tensor_split"], "prime_order": info["prime_order"],
                         "one_group_per_stage": {"scratch_gib": round(info0["scratch_bytes"] / 2**30, 2),
                                                 "kernels": info0["launches"]}},
            "traced_kernels_ms": {k: round(v[1], 3) for k, v in sorted(tr.items(), key=lambda x: -x[1][1])
                                  if k.startswith("k_")}}


SERVE_STEPS = [k for k in range(1, 33)] + [-k for k in range(1, 33)]    # 64 resident rotation keys


def serving_requests(n, rate, levels_lo, levels_hi, seed_index=3):
    """Seeded request stream: Poisson arrivals at `rate` per second, HMult+relin
    and HRotate with probability 1/2 each, levels uniform on [lo, hi], steps
    uniform over the 64 resident rotation keys."""
    st = si.Stream(si.workload_seed(seed_index), 1)
    gaps = -np.log(1.0 - st.unit(n)) / rate
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(n):
        kind = 1 + st.below(2)                        # OP_HMULT = 1, OP_ROTATE = 2
        nl = levels_lo + st.below(levels_hi - levels_lo + 1)
        reqs.append((kind, nl, st.below(1 << 20), SERVE_STEPS[st.below(len(SERVE_STEPS))]))
    return arrivals, reqs


def run_serving(args, ctx, dA, dK, P, scale):
    """Request server under a Poisson stream of HMult+relin / HRotate requests
    at levels 2..30 on a resident pool of 256 ciphertexts, with the
    relinearisation key and 64 rotation keys resident and admission bounded by
    a 120 GB budget for keys + pool + the server's arena.  Reports latency
    percentiles (request submitted -> completion observed), the served rate, a
    closed-loop saturation run, and the same request mix one call per op."""
    import torch

    import paper_2507_04775_gb300 as fides
    N, nq = ctx.N, P.nq
    lo, hi = 2, nq
    # resident keys: 1 relinearisation + 64 rotation keys, separate buffers (120 MiB each)
    rlk = ctx.relin_key(dK[0].clone())
    rot = {k: ctx.rotation_key(dK[1 + i % (len(dK) - 1)].clone(), k) for i, k in enumerate(SERVE_STEPS)}
    # resident operand pool: 256 ciphertexts, levels 2..30 round-robin
    pool_lv = [lo + i % (hi - lo + 1) for i in range(256)]
    pool = [dA[i % len(dA)].view(2, nq, N)[:, :nl].contiguous().view(-1) for i, nl in enumerate(pool_lv)]
    by_level = {}
    for i, nl in enumerate(pool_lv):
        by_level.setdefault(nl, []).append(i)
    resident = (rlk.tensor.numel() + sum(t.tensor.numel() for t in rot.values()) + sum(t.numel() for t in pool)) * 8
    budget = int(args.serve_budget_gb * 1e9)
    arena = budget - resident
    torch.cuda.synchronize()

    def operands(r):
        kind, nl, pick, steps = r
        idx = by_level[nl]
        a = pool[idx[pick % len(idx)]]
        b = pool[idx[(pick + 1) % len(idx)]] if kind == fides.OP_HMULT else None
        return a, b

    srv = fides.Server(ctx, arena, n_lanes=args.serve_lanes, max_batch=args.serve_max_batch)
    srv.set_relin_key(rlk)
    for k, t in rot.items():
        srv.add_rotation_key(k, t)

    def drive(arrivals, reqs, closed_depth=0):
        """Open loop (arrivals) or closed loop (closed_depth outstanding)."""
        done, lag = [], []
        n, i = len(reqs), 0
        outstanding = 0
        t0 = fides.now_ns()
        while len(done) < n:
            now = fides.now_ns()
            if closed_depth:
                while i < n and outstanding < closed_depth:
                    a, b = operands(reqs[i])
                    srv.submit(reqs[i][0], a, reqs[i][1], b=b, steps=reqs[i][3], tag=i, scale_a=scale, scale_b=scale)
                    i += 1
                    outstanding += 1
            else:
                while i < n and now - t0 >= arrivals[i] * 1e9:
                    a, b = operands(reqs[i])
                    srv.submit(reqs[i][0], a, reqs[i][1], b=b, steps=reqs[i][3], tag=i, scale_a=scale, scale_b=scale)
                    lag.append(fides.now_ns() - t0 - arrivals[i] * 1e9)
                    i += 1
                    outstanding += 1
            for c in srv.poll(timeout_us=0):
                if c.status != 0:
                    raise RuntimeError("request %d failed with status %d" % (c.tag, c.status))
                srv.release(c.id)
                done.append(c)
                outstanding -= 1
        return done, lag, t0

    def summary(done, t0, n):
        lat = np.array([c.latency_ns for c in done], dtype=np.float64) / 1e6
        t_end = max(c.t_done_ns for c in done)
        span = (t_end - min(c.t_submit_ns for c in done)) / 1e9
        groups = np.array([c.group_ops for c in done])
        return {"requests": n, "ops_per_s": round(n / span, 1), "seconds": round(span, 3),
                "p50_ms": round(float(np.percentile(lat, 50)), 3), "p90_ms": round(float(np.percentile(lat, 90)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3), "max_ms": round(float(lat.max()), 3),
                "mean_group": round(float(groups.mean()), 2)}

    # warm-up: one request of each kind at a few levels
    wa, wr = serving_requests(64, 1e9, lo, hi, seed_index=4)
    drive(wa, wr)
    st0 = srv.stats()
    arrivals, reqs = serving_requests(args.serve_requests, args.serve_rate, lo, hi)
    done, lag, t0 = drive(arrivals, reqs)
    st1 = srv.stats()
    open_loop = summary(done, t0, len(reqs))
    open_loop["offered_per_s"] = args.serve_rate
    open_loop["client_lag_p99_ms"] = round(float(np.percentile(np.array(lag) / 1e6, 99)), 3)
    open_loop["kernels"] = int(st1["kernel_launches"] - st0["kernel_launches"])
    open_loop["groups"] = int(st1["groups"] - st0["groups"])
    open_loop["device_busy_frac"] = round((st1["device_ms"] - st0["device_ms"]) / 1e3 / open_loop["seconds"], 3)
    open_loop["admission_stalls"] = int(st1["admission_stalls"] - st0["admission_stalls"])

    # saturation: the same mix with many requests outstanding
    n_sat = min(len(reqs), args.serve_saturate)
    sat_done, _, t0s = drive(None, reqs[:n_sat], closed_depth=args.serve_depth)
    saturation = summary(sat_done, t0s, n_sat)
    saturation["outstanding"] = args.serve_depth
    st2 = srv.stats()

    # the same requests, one library call per operation, back to back
    n_plain = min(n_sat, 2000)
    out = torch.empty(2 * nq * N, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def plain(rs):
        for r in rs:
            a, b = operands(r)
            if r[0] == fides.OP_HMULT:
                ctx.hmult(a, b, r[1], rlk, out, scale, scale)
            else:
                ctx.rotate(a, r[1], r[3], rot[r[3]], out, scale)
    plain(reqs[:32])
    torch.cuda.synchronize()
    e0.record(stream)
    plain(reqs[:n_plain])
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ops = n_plain / (e0.elapsed_time(e1) / 1e3)
    srv.close()
    del pool, rot, rlk
    torch.cuda.empty_cache()
    return {"workload": "Poisson %g req/s, HMult+relin / HRotate 50/50, levels uniform {2..30}, 256 resident "
                        "ciphertexts, rlk + 64 rotation keys resident, %g GB budget" % (args.serve_rate, args.serve_budget_gb),
            "lanes": args.serve_lanes, "max_batch": args.serve_max_batch,
            "resident_gb": round(resident / 1e9, 2), "arena_gb": round(arena / 1e9, 2),
            "arena_peak_gb": round(st2["arena_peak"] / 1e9, 3),
            "open_loop": open_loop, "saturation": saturation,
            "plain_ops_per_s": round(plain_ops, 1), "plain_requests": n_plain,
            "latency": "submit to completion observed by the dispatcher (host CLOCK_MONOTONIC)"}


def run_ops(args, ctx, dA, dB, dK, P, scale):
    """The operations beyond the key-switching step, at 30 limbs: 8 hoisted
    rotations against 8 single rotations, a 32-diagonal baby-step giant-step
    linear transform (n1 = 8), and the element-wise kernels against the HBM
    peak (their roofline: bytes read + written per launch)."""
    import torch

    import paper_2507_04775_gb300 as fides
    N, nl = ctx.N, P.nq
    a, b = dA[0], dB[0]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    steps = [1, 2, 3, 4, 5, 6, 7, 8]
    keys = [ctx.rotation_key(dK[1 + i % (len(dK) - 1)], s) for i, s in enumerate(steps)]
    outs = [torch.empty(2 * nl * N, dtype=torch.int64, device="cuda") for _ in steps]
    t_h = timed(lambda: ctx.rotate_hoisted(a, nl, steps, keys, outs, scale), 10)
    t_p = timed(lambda: [ctx.rotate(a, nl, k, key, o, scale) for k, key, o in zip(steps, keys, outs)], 10)
    res["hoisted_rotations"] = {"rotations": len(steps), "limbs": nl, "hoisted_ms": round(t_h, 3),
                                "single_ms": round(t_p, 3), "speedup": round(t_p / t_h, 3)}
    # linear transform: 32 diagonals {0..7} x giant steps {0, 8, 16, 24} -> 7 baby + 3 giant rotations
    idx = list(range(32))
    n1 = 8
    st = si.Stream(si.workload_seed(1), 20)
    pts = [fides.to_device(si.uniform_poly(st, ctx.q, N)) for _ in idx]
    lt_keys = [ctx.rotation_key(dK[1 + (k % (len(dK) - 1))], k)
               for k in sorted({i % n1 for i in idx if i % n1} | {n1 * (i // n1) for i in idx if i // n1})]
    out = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
    words = (7 + 2) * 2 * nl * N
    work = torch.empty(words, dtype=torch.int64, device="cuda")
    t_lt = timed(lambda: ctx.linear_transform(a, nl, idx, pts, n1, lt_keys, out, scale, 1.0, work=work), 5)
    res["linear_transform"] = {"diagonals": len(idx), "n1": n1, "limbs": nl, "ms": round(t_lt, 3),
                               "rotations": "7 hoisted baby steps + 3 giant steps"}
    # element-wise kernels: bytes read + written per launch over the measured HBM peak
    hbm_peak = peaks()[0]
    limb = 8 * N
    pt = pts[0]
    o = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
    ew = {}
    k3 = [3 % q for q in ctx.q[:nl]]
    flush = torch.empty(256 << 20, dtype=torch.int8, device="cuda")     # larger than L2
    for name, fn, nbytes in (
            ("hadd", lambda: ctx.hadd(a, b, nl, o, scale), 6 * nl * limb),
            ("ptmult", lambda: ctx.ptmult(a, pt, nl, o, scale), 5 * nl * limb),
            ("scalar_mult", lambda: ctx.scalar_mult(a, k3, nl, o, scale), 4 * nl * limb),
            ("ptmac_8", lambda: ctx.linear_transform(a, nl, list(range(8)), pts[:8], 8, lt_keys, out, scale, 1.0,
                                                     work=work), None)):
        fn()
        torch.cuda.synchronize()
        fides.trace_reset()
        fides.trace_enable(True)
        for _ in range(20):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        fides.trace_enable(False)
        tr = fides.trace_read()
        kname = "k_ptmac" if name.startswith("ptmac") else "k_elem"
        n_l, ms = tr[kname]
        t = ms / n_l
        if nbytes is None:     # 8 baby-step ciphertexts and 8 plaintexts read, one ciphertext written
            nbytes = (8 * 2 * nl + 8 * nl + 2 * nl) * limb
        gbs = nbytes / (t / 1e3) / 1e9
        ew[name] = {"us": round(t * 1e3, 2), "GB/s": round(gbs, 1), "frac_of_hbm": round(gbs / hbm_peak, 3)}
    del flush
    res["elementwise"] = ew
    # the logN=12 set (3 x 40-bit q, 1 x 50-bit p, dnum 3): latency of one HMult+relin
    S = si.SMALL
    sq = fides.find_primes(S.logN, S.q_bits, S.nq)
    sp = fides.find_primes(S.logN, S.p_bits, S.nk, exclude=sq)
    sctx = fides.Context(S.logN, sq, sp, S.dnum)
    st2 = si.Stream(si.workload_seed(0), 21)
    sa = fides.to_device(np.stack([si.uniform_poly(st2, sq, sctx.N) for _ in range(2)]))
    sb = fides.to_device(np.stack([si.uniform_poly(st2, sq, sctx.N) for _ in range(2)]))
    skey = sctx.relin_key(fides.to_device(np.stack([np.stack([si.uniform_poly(st2, sq + sp, sctx.N)
                                                              for _ in range(2)]) for _ in range(S.dnum)])))
    so = torch.empty_like(sa)
    t_small = timed(lambda: sctx.hmult(sa, sb, S.nq, skey, so), 200)
    l0 = fides.kernel_launches()
    sctx.hmult(sa, sb, S.nq, skey, so)
    torch.cuda.synchronize()
    res["hmult_logN12_L3"] = {"us": round(t_small * 1e3, 2), "launches": int(fides.kernel_launches() - l0),
                              "note": "one call at a time; latency bound (each launch covers 3 to 4 limbs of 32 KiB)"}
    sctx.close()
    # HMult+relin latency at every level of the bench context (one call at a
    # time): the key switch gets cheaper each time a digit is dropped
    rlk = ctx.relin_key(dK[0])
    by_level = {}
    for lv in range(1, nl + 1):
        la = dA[0].view(2, nl, N)[:, :lv].contiguous().view(-1)
        lb = dB[0].view(2, nl, N)[:, :lv].contiguous().view(-1)
        lo = torch.empty(2 * lv * N, dtype=torch.int64, device="cuda")
        by_level[lv] = round(timed(lambda: ctx.hmult(la, lb, lv, rlk, lo, scale, scale), 10) * 1e3, 1)
    res["hmult_us_by_level"] = by_level
    # PtMult followed by Rescale at several levels (the paper's PtMult+Rescale
    # figure, one call of each at a time)
    pr_level = {}
    for lv in (2, 5, 10, 15, 20, 25, 30):
        la = dA[0].view(2, nl, N)[:, :lv].contiguous().view(-1)
        lpt = fides.to_device(si.uniform_poly(st, ctx.q[:lv], N))
        lm = torch.empty(2 * lv * N, dtype=torch.int64, device="cuda")
        lr = torch.empty(2 * (lv - 1) * N, dtype=torch.int64, device="cuda")
        pr_level[lv] = round(timed(lambda: (ctx.ptmult(la, lpt, lv, lm, scale), ctx.rescale(lm, lv, lr, scale)),
                                   20) * 1e3, 1)
    res["ptmult_rescale_us_by_level"] = pr_level
    # HMult+relin at the top level across ring degrees, with sets whose key
    # sizes are those the paper quotes for its parameter-set comparison (2.3,
    # 7.7, 20, 152 and 360 MB; the sets themselves are in a figure whose
    # values the text does not give); logN=16 is the paper's Table III set
    # [2^16, 29, 59, 4] (30 limbs of 59 bits, K = 8)
    by_set = {}
    for logN, L, dnum, qb in ((13, 6, 2, 54), (14, 7, 3, 54), (15, 14, 2, 54), (16, 30, 4, 59), (17, 36, 4, 54)):
        K = -(-L // dnum)
        pq = fides.find_primes(logN, qb, L)
        pp = fides.find_primes(logN, 60, K, exclude=pq)
        pctx = fides.Context(logN, pq, pp, dnum)
        if not args.no_autotune:
            pctx.autotune(2 * (L + K))
        pN = pctx.N
        st3 = si.Stream(si.workload_seed(1), 22 + logN)
        pa = fides.to_device(np.stack([si.uniform_poly(st3, pq, pN) for _ in range(2)]))
        pb = fides.to_device(np.stack([si.uniform_poly(st3, pq, pN) for _ in range(2)]))
        kbuf = fides.to_device(np.stack([np.stack([si.uniform_poly(st3, pq + pp, pN) for _ in range(2)])
                                         for _ in range(dnum)]))
        pk = pctx.relin_key(kbuf)
        po = torch.empty_like(pa)
        t_set = timed(lambda: pctx.hmult(pa, pb, L, pk, po, scale, scale), 20)
        by_set["logN%d_L%d_dnum%d" % (logN, L, dnum)] = {
            "us": round(t_set * 1e3, 1), "K": K, "key_mib": round(kbuf.numel() * 8 / 2 ** 20, 1),
            "ops_per_s": round(1e3 / t_set, 1)}
        pk.close()
        del pa, pb, po, kbuf
        pctx.close()
    res["hmult_by_parameter_set"] = by_set
    # forward + inverse NTT of 32 limbs at every ring degree (butterflies per second)
    by_degree = {}
    for logN in range(12, 18):
        dq = fides.find_primes(logN, 54, 30)
        dp = fides.find_primes(logN, 60, 2, exclude=dq)
        dctx = fides.Context(logN, dq, dp, 3)
        if not args.no_autotune:
            dctx.autotune(32)
        n = 32
        x = fides.to_device(np.concatenate([si.uniform_poly(st2, dq + dp, dctx.N)]))
        t = timed(lambda: (dctx.ntt(x, 0, n), dctx.intt(x, 0, n)), 20)
        bfly = 2 * n * (dctx.N // 2) * logN
        by_degree[logN] = {"us_fwd_inv_32_limbs": round(t * 1e3, 1),
                           "gbutterfly_per_s": round(bfly / (t / 1e3) / 1e9, 1)}
        dctx.close()
    res["ntt_by_degree"] = by_degree
    # forward + inverse NTT at logN=16 by limb count (working set 0.5 MiB per
    # limb): time per limb as the launches grow
    by_limbs = {}
    for n_l in (1, 2, 4, 8, 16, 32, 64, 128):
        per, bat = (n_l, 1) if n_l <= 16 else (16, n_l // 16)   # batches of 16 q-limbs
        x = fides.to_device(np.stack([si.uniform_poly(st2, ctx.q[:per], N) for _ in range(bat)]))
        t = timed(lambda: (ctx.ntt(x, 0, per, bat), ctx.intt(x, 0, per, bat)), 20)
        by_limbs[n_l] = {"us_fwd_inv": round(t * 1e3, 1), "us_per_limb": round(t * 1e3 / n_l, 2),
                         "working_set_mib": n_l * N * 8 / 2 ** 20}
        del x
    res["ntt_logN16_by_limbs"] = by_limbs
    res["elementwise_note"] = ("device time of the kernel (CUDA events around each launch), L2 flushed before each "
                               "launch; 30-limb operands; bytes = operands read + result written once")
    return res


def run_bootstrap(args):
    """Bootstrapping at logN=16 (2^15 slots): q_0 of 60 bits and 29 q_i of 54
    bits, K = 10 special 60-bit primes, dnum = 3; the library's planner builds
    the program (CoeffToSlot / SlotToCoeff with level budget 3/3, EvalMod of
    Chebyshev degree 119 plus 2 double-angle steps).  A batch of 8 one-limb
    ciphertexts is bootstrapped one after another on one stream, then dealt
    over --bootstrap-lanes streams of the same context (one program, with its
    own work buffer, per lane).  Keys and ciphertexts are
    uniform residues of the right shapes (timing only; the decryption check is
    in the GPU tests)."""
    import torch

    import paper_2507_04775_gb300 as fides
    from paper_2507_04775_gb300 import bootstrap as bt
    logN = 16
    q0 = fides.find_primes(logN, 60, 1)
    q = q0 + fides.find_primes(logN, 54, 29, exclude=q0)
    p = fides.find_primes(logN, 60, 10, exclude=q)
    ctx = fides.Context(logN, q, p, 3)
    if not args.no_autotune:
        ctx.autotune(128)
    N = ctx.N
    t0 = time.perf_counter()
    prog = bt.plan(N, q, 2.0 ** 50)
    t_plan = time.perf_counter() - t0
    st = si.Stream(si.workload_seed(4), 30)
    key = fides.to_device(np.stack([np.stack([si.uniform_poly(st, q + p, N) for _ in range(2)]) for _ in range(3)]))
    rks = [ctx.rotation_key(key.clone(), s) for s in prog.rot_steps]
    rlk, ck = ctx.relin_key(key.clone()), ctx.conjugation_key(key.clone())
    t0 = time.perf_counter()
    dp = bt.DeviceProgram(ctx, prog, rlk, ck, rks)
    t_load = time.perf_counter() - t0
    cts = [fides.to_device(np.stack([si.uniform_poly(st, q[:1], N) for _ in range(2)]))
           for _ in range(args.bootstrap_batch)]
    outs = [torch.empty(2 * dp.out_limbs * N, dtype=torch.int64, device="cuda") for _ in cts]
    stream = torch.cuda.current_stream()
    launches0 = fides.kernel_launches()
    dp.run(cts[0], outs[0], 2.0 ** 50)
    torch.cuda.synchronize()
    per_boot_launches = fides.kernel_launches() - launches0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for c, o in zip(cts, outs):
        dp.run(c, o, 2.0 ** 50)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_one = e0.elapsed_time(e1)
    # the same batch over several lanes: one program (own work buffer) per
    # stream of the same context, ciphertexts dealt round robin; the events
    # on the launching stream bracket every lane (each lane waits on e0 and
    # e1 waits on each lane)
    lanes = max(1, args.bootstrap_lanes)
    ms = ms_one
    if lanes > 1:
        dps = [dp] + [bt.DeviceProgram(ctx, prog, rlk, ck, rks) for _ in range(lanes - 1)]
        sts = [torch.cuda.Stream() for _ in range(lanes)]
        for k in range(lanes):      # warm every program once
            dps[k].run(cts[k % len(cts)], outs[k % len(cts)], 2.0 ** 50, stream=sts[k])
        torch.cuda.synchronize()
        e0.record(stream)
        for s_ in sts:
            s_.wait_event(e0)
        for k, (c, o) in enumerate(zip(cts, outs)):
            dps[k % lanes].run(c, o, 2.0 ** 50, stream=sts[k % lanes])
        for s_ in sts:
            ev = torch.cuda.Event()
            ev.record(s_)
            stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        for d_ in dps[1:]:
            d_.close()
    # one more bootstrap with every operation and kernel bracketed by events
    fides.trace_reset()
    fides.trace_enable(True)
    dp.run(cts[0], outs[0], 2.0 ** 50)
    torch.cuda.synchronize()
    fides.trace_enable(False)
    tr = fides.trace_read()
    fides.trace_reset()
    top_ops = {k[3:]: [v[0], round(v[1], 2)] for k, v in sorted(tr.items(), key=lambda x: -x[1][1])
               if k.startswith("op_") and k != "op_program"}
    kern = {k: [v[0], round(v[1], 2)] for k, v in sorted(tr.items(), key=lambda x: -x[1][1]) if k.startswith("k_")}
    # sparse packing at the slot counts of the paper's Table IV below 2^15:
    # the same batch on one stream (a trace of rotate-and-add steps after
    # ModRaise, then slots-point transforms)
    sparse = {}
    for slots in (1 << 14, 512, 64):
        t0 = time.perf_counter()
        sp = bt.plan(N, q, 2.0 ** 50, slots=slots)
        t_sp = time.perf_counter() - t0
        srks = [ctx.rotation_key(key.clone(), s) for s in sp.rot_steps]
        sdp = bt.DeviceProgram(ctx, sp, rlk, ck, srks)
        souts = [torch.empty(2 * sdp.out_limbs * N, dtype=torch.int64, device="cuda") for _ in cts]
        sdp.run(cts[0], souts[0], 2.0 ** 50)
        torch.cuda.synchronize()
        e0.record(stream)
        for c, o in zip(cts, souts):
            sdp.run(c, o, 2.0 ** 50)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_s = e0.elapsed_time(e1)
        sparse[str(slots)] = {"ms_per_ciphertext": round(ms_s / len(cts), 2), "one_lane_ms_per_batch": round(ms_s, 2),
                              "limbs_out": sdp.out_limbs, "rotation_keys": len(sp.rot_steps),
                              "trace_rotations": sum(1 for ins in sp.instr if ins[0] == bt.OP["ROT"]),
                              "plan_s": round(t_sp, 1)}
        sdp.close()
        del srks, souts
    counts = {}
    for ins in prog.instr:
        counts[ins[0]] = counts.get(ins[0], 0) + 1
    names = {v: k for k, v in bt.OP.items()}
    res = {"workload": "bootstrap logN=16, 2^15 slots, L=30 (1 x 60-bit + 29 x 54-bit), K=10, dnum=3, "
                       "CtS/StC level budget 3/3, EvalMod Chebyshev degree 119 + 2 double angles, batch of %d" % len(cts),
           "ms_per_ciphertext": round(ms / len(cts), 2), "ms_per_batch": round(ms, 2), "batch": len(cts),
           "lanes": lanes, "one_lane_ms_per_batch": round(ms_one, 2),
           "limbs_out": dp.out_limbs, "rotation_keys": len(prog.rot_steps),
           "plaintexts": sum(len(t["coeffs"]) for t in prog.lts), "instructions": len(prog.instr),
           "instruction_mix": {names[k]: v for k, v in sorted(counts.items())},
           "kernels_per_bootstrap": int(per_boot_launches), "device_buffers": dp.buffers,
           "work_gib": round(dp.work_words * 8 / 2 ** 30, 2), "plan_s": round(t_plan, 1), "load_s": round(t_load, 1),
           "traced_ops_calls_ms": top_ops, "traced_kernels_launches_ms": kern,
           "traced_note": "one traced bootstrap; nested operations (a linear transform's rotations) count in both",
           "one_lane_ms_per_ciphertext": round(ms_one / len(cts), 2),
           "sparse_slots": sparse}
    dp.close()
    del rks, cts, outs, key
    ctx.close()
    torch.cuda.empty_cache()
    return res


def run_ops_only(args, local):
    import torch

    import paper_2507_04775_gb300 as fides
    torch.cuda.set_device(local)
    P = si.FULL
    q = fides.find_primes(P.logN, P.q_bits, P.nq)
    p = fides.find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    ctx = fides.Context(P.logN, q, p, P.dnum)
    A, B, keys = workload_inputs(P, q, p, si.workload_seed(1))
    dA = [fides.to_device(x) for x in A]
    dB = [fides.to_device(x) for x in B]
    dK = [fides.to_device(x) for x in keys]
    return {"ops": run_ops(args, ctx, dA, dB, dK, P, 2.0 ** P.log_scale)}


def load_traffic(kernel, bytes_per_launch):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = t.get(kernel)
    if not ent or ent.get("sources_sha") != sources_sha(kernel):
        return None
    # the capture ran a smaller case: scale by the units one bench launch processes
    return int(ent["dram_bytes_per_unit"] * bytes_per_launch / ent["algorithmic_bytes_per_unit"])


KERNEL_SOURCES = {"k_ntt": ["ntt.cuh", "ntt_impl.cuh", "ntt_l16.cu", "fides_internal.cuh"],
                  "k_bconv_tc": ["bconv_tc.cuh", "kernels.cuh", "fides_internal.cuh"],
                  "k_bconv": ["kernels.cuh", "fides_internal.cuh"],
                  "k_inner": ["kernels.cuh", "fides_internal.cuh"]}


def sources_sha(kernel: str = "k_ntt") -> str:
    """Hash of the sources a kernel is compiled from (a DRAM-traffic figure
    measured on other sources is stale)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2507_04775_gb300", "csrc")
    files = next((v for k, v in KERNEL_SOURCES.items() if kernel.startswith(k)), None)
    for f in sorted(files or [f for f in os.listdir(d) if f.endswith((".cu", ".cuh"))]):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def run_e2e(args, world, ctx, A, B, rlk, rks, nl, N, scale):
    """Same steps through the public API with host buffers: every step copies
    its input pair from pinned host memory and reads its two results back
    (the rescaled product and the rotation; the unrescaled product stays on
    the device as the intermediate it is).  Copies run on their own streams
    over three buffer slots, so the input copy of step k+1 and the output copy
    of step k-1 overlap the compute of step k (the input copy of a slot waits
    only for the output copy of three steps before).  Also reported: the host
    time to issue a step, and the time per step of the same copies alone."""
    import gc
    import torch
    steps = max(5, min(args.steps, 200))
    hA = [torch.from_numpy(x.view(np.int64).reshape(-1)).pin_memory() for x in A]
    hB = [torch.from_numpy(x.view(np.int64).reshape(-1)).pin_memory() for x in B]

    def dev(words):
        return torch.empty(words, dtype=torch.int64, device="cuda")

    w_in, w_rs = 2 * nl * N, 2 * (nl - 1) * N
    slots = []
    NSLOT = 3
    for _ in range(NSLOT):
        slots.append({"a": dev(w_in), "b": dev(w_in), "m": dev(w_in), "r": dev(w_in), "s": dev(w_rs),
                      "hr": torch.empty(w_in, dtype=torch.int64).pin_memory(),
                      "hs": torch.empty(w_rs, dtype=torch.int64).pin_memory(),
                      "in_ready": torch.cuda.Event(), "computed": torch.cuda.Event(), "drained": torch.cuda.Event()})
    comp, h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def step(k, compute=True):
        sl, i = slots[k % NSLOT], k % POOL
        with torch.cuda.stream(h2d):
            h2d.wait_event(sl["drained"])          # outputs of step k-3 copied out, inputs consumed
            sl["a"].copy_(hA[i], non_blocking=True)
            sl["b"].copy_(hB[i], non_blocking=True)
            sl["in_ready"].record(h2d)
        if compute:
            with torch.cuda.stream(comp):
                comp.wait_event(sl["in_ready"])
                s = ctx.hmult(sl["a"], sl["b"], nl, rlk, sl["m"], scale, scale, stream=comp)
                ctx.rescale(sl["m"], nl, sl["s"], s, stream=comp)
                ctx.rotate(sl["a"], nl, 1 << (k % N_ROT), rks[k % N_ROT], sl["r"], scale, stream=comp)
                sl["computed"].record(comp)
        else:
            sl["computed"].record(h2d)
        with torch.cuda.stream(d2h):
            d2h.wait_event(sl["computed"])
            sl["hs"].copy_(sl["s"], non_blocking=True)
            sl["hr"].copy_(sl["r"], non_blocking=True)
            sl["drained"].record(d2h)

    for sl in slots:
        sl["drained"].record(d2h)
    for k in range(3):
        step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the host loop issues every step ahead of the device; a collection of
    # the interpreter's garbage in the middle of it would leave the device
    # idle, so it runs before the timed region and not inside it (as timeit
    # does)
    gc.collect()
    gc_was = gc.isenabled()
    gc.disable()
    barrier(world)
    torch.cuda.synchronize()
    e0.record(h2d)
    t0 = time.perf_counter()
    for k in range(steps):
        step(k)
    host_ms = (time.perf_counter() - t0) * 1e3
    d2h.synchronize()
    e1.record(d2h)
    torch.cuda.synchronize()
    if gc_was:
        gc.enable()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    # the same copies without the compute (what the copies alone would allow)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    c0.record(h2d)
    for k in range(steps):
        step(k, compute=False)
    d2h.synchronize()
    c1.record(d2h)
    torch.cuda.synchronize()
    h2d_b, d2h_b = 2 * hA[0].numel() * 8, (w_in + w_rs) * 8
    copy_ms = c0.elapsed_time(c1) / steps
    return {"value": round(2 * steps * world / (ms / 1e3), 2), "unit": "ops/s", "steps": steps,
            "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
            "ms_per_step": round(ms / steps, 4),
            "host_issue_ms_per_step": round(host_ms / steps, 4),
            "copies_alone_ms_per_step": round(copy_ms, 4),
            "copies_alone_gbs": round((h2d_b + d2h_b) / (copy_ms / 1e3) / 1e9, 1),
            "pipelined": "input copies, compute and result copies on three streams, three buffers deep"}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_steps(P, q, p, A, B, keys, budget_s, max_steps):
    import oracle
    ctx = oracle.Context(P.logN, q, p, P.dnum)
    done, t0 = 0, time.perf_counter()
    while done < max_steps:
        i = done % len(A)
        out = ctx.hmult(A[i], B[i], keys[0])
        ctx.rescale(out)
        ctx.rotate(A[i], 1 << (done % N_ROT), keys[1 + done % (len(keys) - 1)])
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return done, time.perf_counter() - t0


def small_inputs():
    """The logN=12 workload (3 x 40-bit q, 1 x 50-bit p, dnum=3): two ciphertext
    pairs, a relinearisation key and two rotation keys, from its own seed."""
    import oracle
    P = si.SMALL
    q = oracle.find_primes(P.logN, P.q_bits, P.nq)
    p = oracle.find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    st = si.Stream(si.workload_seed(0), 10)
    N = 1 << P.logN
    A = [np.stack([si.uniform_poly(st, q, N) for _ in range(2)]) for _ in range(2)]
    B = [np.stack([si.uniform_poly(st, q, N) for _ in range(2)]) for _ in range(2)]
    keys = [np.stack([np.stack([si.uniform_poly(st, q + p, N) for _ in range(2)]) for _ in range(P.dnum)])
            for _ in range(3)]
    return P, q, p, A, B, keys


def cpu_baseline(P, q, p, A, B, keys, budget_s):
    """The oracle as it stands, on the host cores: the bench workload with the
    OpenMP loops on every core (the headline `value`) and on one thread, and
    the logN=12 workload on both."""
    import oracle
    cores = oracle.set_threads(0)
    done, el = oracle_steps(P, q, p, A, B, keys, budget_s, 1000)
    res = {"value": round(2 * done / el, 4), "unit": "ops/s", "cores": cores, "kind": "oracle",
           "sample": "%d step(s) of the same workload (HMult+relin, Rescale, HRotate at 30 limbs), %.1f s" % (done, el)}
    oracle.set_threads(1)
    try:
        d1, e1 = oracle_steps(P, q, p, A, B, keys, 0.0, 1)
        res["single_thread"] = {"value": round(2 * d1 / e1, 4), "unit": "ops/s", "cores": 1,
                                "sample": "%d step of the same workload, %.1f s" % (d1, e1)}
        Ps, qs, ps, As, Bs, Ks = small_inputs()
        small = {"workload": "HMult+relin, Rescale, HRotate of one logN=12 pair (3 x 40-bit q, 1 x 50-bit p, "
                             "dnum=3)", "unit": "ops/s"}
        for n in (1, cores):
            oracle.set_threads(n)
            ds, es = oracle_steps(Ps, qs, ps, As, Bs, Ks, 1.5, 10000)
            small["cores_%d" % n] = {"value": round(2 * ds / es, 2), "cores": n,
                                     "sample": "%d steps, %.2f s" % (ds, es)}
        res["small_config"] = small
    finally:
        oracle.set_threads(cores)
    return res


def run_reference(args, world, rank):
    if rank != 0:
        return None
    P = si.FULL
    import oracle
    q = oracle.find_primes(P.logN, P.q_bits, P.nq)
    p = oracle.find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    A, B, keys = workload_inputs(P, q, p, si.workload_seed(1))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    oracle_steps(P, q, p, A, B, keys, 0.0, min(args.warmup, 1))
    # each step is the full workload step; the number timed is capped so the
    # run stays within a few minutes
    cap = max(1, min(args.steps, 40))
    done, el = oracle_steps(P, q, p, A, B, keys, 120.0, cap)
    value = 2 * done / el
    return {"metric": METRIC, "value": round(value, 4), "unit": "ops/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(el / done * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": workload_config(P, world),
            "cpu_baseline": {"value": round(value, 4), "unit": "ops/s", "cores": cores, "kind": "oracle",
                             "sample": "%d of %d steps timed (capped at 40 steps / 120 s)" % (done, args.steps)},
            "e2e": {"value": round(value, 4), "unit": "ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.ops_only:
        res = run_ops_only(args, local)
    elif args.bootstrap_only:
        import torch
        torch.cuda.set_device(local)
        res = run_bootstrap(args)
    elif args.impl == "reference":
        res = run_reference(args, world, rank)
    else:
        res = run_fides(args, world, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
