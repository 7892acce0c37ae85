#!/usr/bin/env python
"""Benchmark of the Mod-PP-MM hot path on the PC-MM n=4096 workload.

Workload (one step): row-format PC-MM with d = kct = N = 4096 and L = 3 RNS
primes of 50 bits: U (4096 x 4096, N(0,1) quantised to int8 with scale 2^5)
times the a-part and the b-part of 4096 ciphertexts of ring degree 4096, i.e.
six exact Mod-PP-MMs C = U * X mod q_j.  The ciphertexts are row-format RLWE
encryptions of a message matrix M uniform in [-1, 1] at scale 2^40 (ternary
secret, rounded Gaussian error of width 3.2); the line reports the decrypted
result's error against the FP64 product U*M.

Metric: exact Mod-PP-MM throughput in TOPS, counting 2*d*k*n multiply-adds
mod q per (prime, part) plane (so one step is 2 * 4096^3 * 6 = 8.2e11 ops).
Also reported: PC-MM time, cuBLAS FP64 DGEMM time for U*M at the same n and
the ratio ("slowdown vs FP64 matmul"), the FP64-limb path (Strategy 1 on
cuBLAS DGEMM) and its fraction of the measured DGEMM rate, the roofline of
the dominant kernel, an end-to-end number with host buffers, and the CPU
oracle as a baseline.  After the line's own timed region the default run also
measures the rest of the metric as sub-objects of the same line: "config1"
(the 256^3 one-prime product: launch latency in microseconds), "pcmm16384"
(PC-MM n=16384, L=4) and "ccmm" (CC-MM n=8192, Alg. 8, with real keys; stage
split, slowdown vs the 8192^3 DGEMM, decrypted error, CRT GEMM roofline).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs the same workload on its own GPU (independent
replicas, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("PC-MM/CC-MM time and slowdown vs FP64 matmul, same n, 1 GB300; "
          "exact Mod-PP-MM TOPS")
UNIT = "TOPS"
D = K = N = 4096  # overridden by --n (profiling of smaller cases only)
NPRIMES = 3
PRIME_BITS = 50
SEED = 2024
WORKLOAD = ("PC-MM n=4096: U 4096x4096 int8 (N(0,1)*2^5) x row-RLWE ciphertext matrix "
            "4096 cts of degree 4096 (encryptions of M uniform in [-1,1] at scale 2^40), L=3 primes "
            "of 50 bits, a- and b-part (6 Mod-PP-MM planes)")


# DRAM bytes (read + write) of one gemm_f16_kernel launch of this workload, from
# one ncu capture of the current kernel: 1264641536 read + 791442432 written.
GEMM_TRAFFIC_N4096 = 1264641536 + 791442432


def mod_ops_per_step() -> float:
    return 2.0 * D * K * N * 2 * NPRIMES


# ----------------------------------------------------------------- helpers

def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(elapsed_ms: float, device) -> float:
    """The slowest rank's timed-region length (the job's time); every rank
    gets it.  One rank: unchanged."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: float, steps: int, world: int, max_ms: float) -> float:
    """Units all ranks processed (replicas: each rank runs the whole
    workload) per second of the slowest rank, in tera-units."""
    return units_per_step * steps * world / (max_ms * 1e-3) / 1e12


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region.  start() returns once the first sample has arrived (or after 3 s),
    so that sampling covers the region that follows; samples come every 50 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.reader = None
        self.t_mark = None

    def start(self):
        import threading
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        first = threading.Event()

        def read():
            for line in self.proc.stdout:
                self.lines.append((time.perf_counter(), line))
                first.set()
        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()
        first.wait(3.0)

    def mark(self):
        """Start of the timed region: samples before it are dropped, except the
        last one (the clock state the region starts in)."""
        self.t_mark = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        if self.reader is not None:
            self.reader.join(timeout=5)
        rows = self.lines
        if self.t_mark is not None:
            before = [r for r in rows if r[0] < self.t_mark]
            rows = before[-1:] + [r for r in rows if r[0] >= self.t_mark]
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, line in rows:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def tensor_peak(peaks: dict, region_ms: float):
    """Measured bf16 dense peak that a kernel timed in a region of region_ms
    is held to: the burst figure for a region shorter than one second (the
    clocks stay at their maximum), the sustained one (seconds under the power
    cap) for longer regions.  f16 runs at the bf16 rate on kind::f16."""
    if region_ms < 1000.0:
        return peaks["bf16_tflops"], "burst"
    return peaks["bf16_tflops_sustained"], "sustained"


DELTA = 2.0 ** 40     # CKKS scale of the encrypted message matrix
DEC_TOL = 2.0 ** -20  # decoded-error tolerance, relative to the scale


def _mul_pow2_mod(r, bits: int, q: int):
    """(r * 2^bits) mod q for int64 residues 0 <= r < q < 2^60, in steps of at
    most 3 bits so every intermediate product stays below 2^63."""
    import torch
    while bits > 0:
        k = min(3, bits)
        r = torch.remainder(r * (1 << k), q)
        bits -= k
    return r


def negacyclic_matrix(s, dtype):
    """The N x N matrix S of a ring element s of Z[X]/(X^N + 1): the row vector
    of x's coefficients times S is the coefficient vector of x*s."""
    import torch
    n = s.shape[0]
    j = torch.arange(n, device=s.device)
    diff = j[None, :] - j[:, None]                      # l - j
    S = s[torch.remainder(diff, n)].to(dtype)
    return torch.where(diff >= 0, S, -S)


def negacyclic_rows_mod(X, S, q: int, limb_bits: int = 12):
    """Rows of X (R x N int64 residues mod q < 2^60) times the small ring
    element whose negacyclic matrix is S, modulo q.

    Harness arithmetic for encrypting, key generation and decryption (plain
    PyTorch): X is cut into limb_bits-bit limbs, each limb times S is one
    floating-point matrix product whose sums are integers of magnitude below
    2^limb_bits * N * max|s| (exact: below 2^53 for FP64 S, below 2^24 for
    FP32 S, whose products run as TF32 with limbs of at most 10 bits), and the
    limb products are recombined by Horner steps modulo q in int64."""
    import torch
    nl = -(-int(q).bit_length() // limb_bits)
    mask = (1 << limb_bits) - 1
    tf32 = S.dtype == torch.float32
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = tf32
    try:
        r = torch.zeros(X.shape, dtype=torch.int64, device=X.device)
        for i in reversed(range(nl)):
            limb = ((X >> (limb_bits * i)) & mask).to(S.dtype)
            P = torch.matmul(limb, S).to(torch.int64)
            del limb
            r = torch.remainder(_mul_pow2_mod(r, limb_bits, q) + P, q)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    return r


def make_inputs(seed=SEED, with_message=False):
    """U (int8), the a-parts A (uniform mod q_j) and the b-parts
    B = -A*s + round(Delta*M) + e (mod q_j) of row-format RLWE encryptions of a
    message matrix M uniform in [-1, 1]: ciphertext t encrypts row t of M
    under a ternary secret s with rounded-Gaussian error (sigma = 3.2)."""
    import numpy as np
    import torch
    from paper_2503_16080_gb300 import synth
    primes = synth.ntt_primes(PRIME_BITS, NPRIMES)
    U = synth.quantised_normal_int8(seed, 1, (D, K))
    A = np.stack([synth.uniform_mod(seed, 10 + j, (K, N), q) for j, q in enumerate(primes)])
    M = synth.uniform_unit(seed, 30, (K, N))
    sec = synth.ternary(seed, 31, N)
    e = synth.rounded_gaussian(seed, 32, (K, N))
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() \
        else torch.device("cpu")
    S = negacyclic_matrix(torch.from_numpy(sec).to(dev), torch.float64)
    me = torch.from_numpy(np.floor(M * DELTA + 0.5).astype(np.int64) + e).to(dev)
    B = np.empty_like(A)
    for jq, q in enumerate(primes):
        a_s = negacyclic_rows_mod(torch.from_numpy(A[jq].view(np.int64)).to(dev), S, q)
        B[jq] = torch.remainder(me - a_s, q).cpu().numpy().view(np.uint64)
    del me, S
    if with_message:
        return primes, U, A, B, M, sec
    return primes, U, A, B


def _precision_bits(want, err: float) -> float:
    """Relative precision in bits, log2 max|M| - log2 max|M - M~| (the paper's
    measure, Sec. 6), over the sampled entries."""
    import math
    import numpy as np
    top = float(np.max(np.abs(want)))
    return math.log2(top) - math.log2(err) if err > 0 and top > 0 else float("inf")


def decrypt_error(U, M, sec, Aout, Bout, primes, rows: int = 64):
    """Decrypts sampled rows of (U*A, U*B) with the secret, lifts each
    coefficient by CRT over q_0 q_1 to a centred integer, checks q_2 agrees,
    decodes by 1/Delta and compares with the FP64 product U*M."""
    import numpy as np
    import torch
    dev = Aout.device
    idx = np.unique(np.linspace(0, Aout.shape[1] - 1, rows).astype(np.int64))
    S = negacyclic_matrix(torch.from_numpy(sec).to(dev), torch.float64)
    dec = []
    for jq, q in enumerate(primes):
        sel = torch.from_numpy(idx).to(dev)
        xa = Aout[jq].view(torch.int64).index_select(0, sel)
        xb = Bout[jq].view(torch.int64).index_select(0, sel)
        dec.append(torch.remainder(negacyclic_rows_mod(xa, S, q) + xb, q).cpu().numpy())
    q0, q1 = int(primes[0]), int(primes[1])
    r0 = dec[0].astype(object)
    r1 = dec[1].astype(object)
    x = r0 + q0 * (((r1 - r0) * pow(q0, -1, q1)) % q1)
    half = q0 * q1 // 2
    x = np.where(x > half, x - q0 * q1, x)
    agree = all(np.array_equal((x % int(q)).astype(np.uint64), dec[jq].astype(np.uint64))
                for jq, q in enumerate(primes) if jq >= 2)
    got = x.astype(np.float64) / DELTA
    want = U[idx].astype(np.float64) @ M
    err = float(np.max(np.abs(got - want)))
    return {"rows_sampled": int(len(idx)), "max_abs_err": err, "tolerance": DEC_TOL,
            "precision_bits": _precision_bits(want, err),
            "within_tolerance": err <= DEC_TOL, "other_primes_agree": bool(agree),
            "reference": "FP64 U*M (numpy) on the same rows"}


def _switching_keys(s_old, S32, prp, seed: int, stream: int, L: int, dnum: int):
    """Switching keys s_old[r] -> s for every row r of s_old (count x N small
    int64), in the library's key layout [count, dnum, 2, L+K, N] (digit, part
    a/b, prime): a uniform, b = e - a*s + P s_old on the primes of the digit
    (the RNS gadget of dnum digits of consecutive chain primes), with P the
    product of the K special primes prp[L:]."""
    import torch
    from paper_2503_16080_gb300 import synth
    count, n = s_old.shape
    Lp = len(prp)
    alpha = -(-L // dnum)
    dev = s_old.device
    keys = torch.empty((count, dnum, 2, Lp, n), dtype=torch.uint64, device=dev)
    kv = keys.view(torch.int64)
    e = synth.rounded_gaussian_torch(seed, stream + 90, (count * dnum, n), dev)
    for k, q in enumerate(prp):
        a = synth.uniform_mod_torch(seed, stream + k, (count * dnum, n), q, dev).view(torch.int64)
        kv[:, :, 0, k, :] = a.view(count, dnum, n)
        b = torch.remainder(e.to(torch.int64) - negacyclic_rows_mod(a, S32, q, 10), q)
        del a
        b = b.view(count, dnum, n)
        if k < L:  # |P mod q| < 2^50 and |s_old| <= N <= 2^13: the product fits int64
            Pq = 1
            for p in prp[L:]:
                Pq = Pq * (int(p) % int(q)) % int(q)
            d = k // alpha
            b[:, d, :] = torch.remainder(b[:, d, :] + Pq * s_old, q)
        kv[:, :, 1, k, :] = b
        del b
    return keys


def ccmm_inputs(n: int, primes, prp, dev, seed: int = SEED, dnum=None):
    """Real CKKS inputs for CC-MM at ring degree n (plain PyTorch harness):
    a ternary secret s; column-wise encryptions of M1 and M2 (uniform in
    [-1, 1], scale 2^40; ciphertext j encrypts column j); the automorphism
    keys (slot j switches s(X^(2j+1)) -> s) and the relinearisation key
    (s^2 -> s) for the gadget of dnum digits (default one per chain prime)
    and the special primes prp[len(primes):].  The negacyclic products by s
    run as TF32 matrix products of 10-bit limbs (exact: every sum is an
    integer below 2^24), checked on two rows against the FP64 form."""
    import numpy as np
    import torch
    from paper_2503_16080_gb300 import synth
    L = len(primes)
    dnum = L if dnum is None else dnum
    s = torch.from_numpy(synth.ternary(seed, 800, n)).to(dev)
    S32 = negacyclic_matrix(s, torch.float32)
    probe = synth.uniform_mod_torch(seed, 801, (2, n), prp[-1], dev).view(torch.int64)
    if not torch.equal(negacyclic_rows_mod(probe, S32, prp[-1], 10),
                       negacyclic_rows_mod(probe, negacyclic_matrix(s, torch.float64), prp[-1])):
        raise RuntimeError("TF32 limb products are not exact on this device")

    def encrypt_columns(M, stream):
        ct = torch.empty((2, L, n, n), dtype=torch.uint64, device=dev)
        cv = ct.view(torch.int64)
        me = torch.floor(M.t() * DELTA + 0.5).to(torch.int64)
        me += synth.rounded_gaussian_torch(seed, stream + 50, (n, n), dev).to(torch.int64)
        for j, q in enumerate(primes):
            a = synth.uniform_mod_torch(seed, stream + j, (n, n), q, dev).view(torch.int64)
            cv[0, j] = a
            cv[1, j] = torch.remainder(me - negacyclic_rows_mod(a, S32, q, 10), q)
        return ct

    M1 = synth.uniform_unit_torch(seed, 810, (n, n), dev)
    M2 = synth.uniform_unit_torch(seed, 811, (n, n), dev)
    ct1, ct2 = encrypt_columns(M1, 500), encrypt_columns(M2, 600)
    c = torch.arange(n, device=dev)
    pos = torch.remainder(c[None, :] * (2 * c[:, None] + 1), 2 * n)
    sign = torch.where(pos < n, 1, -1).to(torch.int64)
    s_aut = torch.zeros((n, n), dtype=torch.int64, device=dev)
    s_aut.scatter_(1, torch.remainder(pos, n), sign * s[None, :])
    del pos, sign
    keys = _switching_keys(s_aut, S32, prp, seed, 300, L, dnum)
    del s_aut
    s2 = torch.matmul(s.to(torch.float64)[None, :], negacyclic_matrix(s, torch.float64))
    rkey = _switching_keys(s2.to(torch.int64), S32, prp, seed, 400, L, dnum)
    return {"s": s, "S32": S32, "M1": M1, "M2": M2, "ct1": ct1, "ct2": ct2, "keys": keys,
            "rkey": rkey}


def ccmm_decrypt_error(inp, out, primes, cols: int = 64):
    """Decrypts sampled ciphertexts (columns) of the CC-MM output, lifts by CRT
    over q_0 q_1 (q_2 checked), decodes at scale Delta^2 / q_{L-1} and compares
    with the FP64 product M1 * M2 on the same columns."""
    import numpy as np
    import torch
    n = out.shape[2]
    Lo = out.shape[1]
    idx = np.unique(np.linspace(0, n - 1, cols).astype(np.int64))
    sel = torch.from_numpy(idx).to(out.device)
    ov = out.view(torch.int64)
    dec = []
    for k in range(Lo):
        q = int(primes[k])
        xa = ov[0, k].index_select(0, sel)
        xb = ov[1, k].index_select(0, sel)
        dec.append(torch.remainder(negacyclic_rows_mod(xa, inp["S32"], q, 10) + xb, q)
                   .cpu().numpy())
    q0, q1 = int(primes[0]), int(primes[1])
    r0, r1 = dec[0].astype(object), dec[1].astype(object)
    x = r0 + q0 * (((r1 - r0) * pow(q0, -1, q1)) % q1)
    x = np.where(x > q0 * q1 // 2, x - q0 * q1, x)
    agree = all(np.array_equal((x % int(primes[k])).astype(np.uint64), dec[k].astype(np.uint64))
                for k in range(2, Lo))
    scale = DELTA * DELTA / float(primes[len(primes) - 1])
    got = x.astype(np.float64) / scale
    want = torch.matmul(inp["M1"], inp["M2"].index_select(1, sel)).t().cpu().numpy()
    err = float(np.max(np.abs(got - want)))
    return {"cols_sampled": int(len(idx)), "max_abs_err": err, "tolerance": DEC_TOL,
            "precision_bits": _precision_bits(want, err),
            "within_tolerance": err <= DEC_TOL, "other_primes_agree": bool(agree),
            "scale": "Delta^2 / q_3", "reference": "FP64 M1*M2 (cuBLAS) on the same columns"}


# ----------------------------------------------------------------- CPU oracle

def oracle_rate(U, A, B, primes, target_s: float = 12.0):
    """Times the CPU oracle on a bounded row sample of the same workload and
    returns (TOPS, seconds, rows, threads)."""
    import numpy as np
    import oracle
    oracle.build()
    rows = 2
    U32 = U.astype(np.int32)
    while True:
        sel = np.arange(rows)
        t0 = time.perf_counter()
        oracle.mod_pp_mm_rows(U32, A, primes, sel)
        oracle.mod_pp_mm_rows(U32, B, primes, sel)
        dt = time.perf_counter() - t0
        if dt >= target_s / 4 or rows >= 512:
            break
        rows = min(512, max(rows * 2, int(rows * target_s / 4 / max(dt, 1e-3))))
    ops = 2.0 * rows * K * N * 2 * len(primes)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return ops / dt / 1e12, dt, rows, threads


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    primes, U, A, B = make_inputs()
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        tops, dt, rows, threads = oracle_rate(U, A, B, primes, target_s=max(2.0, 20.0 / (args.steps + args.warmup)))
        if i >= args.warmup:
            vals.append(tops)
            info = (dt, rows, threads)
    value = statistics.median(vals)
    dt, rows, threads = info
    sample = (f"{rows} of {D} output rows of each of the 6 planes (a-part and b-part, 3 primes), "
              f"full k={K} and n={N}; rate extrapolates linearly in rows")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": mod_ops_per_step() / (value * 1e12) * 1e3,
            "ms_per_step_extrapolated": True,
            "ms_per_step_note": (f"a whole step extrapolated from the timed {rows}-row sample "
                                 f"({dt * 1e3:.0f} ms of wall time per sample step)"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "d": D, "k": K, "N": N,
                                            "primes": NPRIMES, "prime_bits": PRIME_BITS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- GPU arm

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_info()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16080_gb300 as pkg

    if args.digit_bits:
        pkg.set_digit_bits(args.digit_bits)
    primes, U_np, A_np, B_np, M_np, sec = make_inputs(with_message=True)
    U = torch.from_numpy(U_np).to(dev)
    A = torch.from_numpy(A_np).to(dev)
    B = torch.from_numpy(B_np).to(dev)
    Aout = torch.empty((NPRIMES, D, N), dtype=torch.uint64, device=dev)
    Bout = torch.empty_like(Aout)
    stream = torch.cuda.current_stream()

    def step():
        pkg.pc_mm(U, A, B, primes, out=(Aout, Bout))

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if pkg.last_status() != 0:
        raise RuntimeError("device status word set during warm-up")

    clocks = ClockSampler(local)
    clocks.start()
    pkg.profile_enable(True)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    elapsed_ms = e0.elapsed_time(e1)
    gemm_ms, gemm_n = pkg.profile_read(pkg.KERNEL_GEMM)
    split_ms, split_n = pkg.profile_read(pkg.KERNEL_SPLIT)
    u16_ms, u16_n = pkg.profile_read(pkg.KERNEL_U16)
    pkg.profile_enable(False)
    clk = clocks.stop()
    if pkg.last_status() != 0:
        raise RuntimeError("device status word set during the timed region")

    max_ms = max_over_ranks(elapsed_ms, dev)
    ms_per_step = max_ms / args.steps
    value = whole_job_rate(mod_ops_per_step(), args.steps, ws, max_ms)

    line = None
    if rank == 0 and args.quick:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "quick": True,
                "gemm_ms_per_step": gemm_ms / args.steps, "split_ms_per_step": split_ms / args.steps,
                "launches_per_step": (gemm_n + split_n + u16_n) / args.steps,
                "u16_avg_ms": u16_ms / max(u16_n, 1), "n": N, "digit_bits": pkg.get_digit_bits()}
    elif rank == 0:
        peaks, peak_src = load_peaks()
        digits = pkg.plan_info(K, primes[0])["digits"]
        planes = 2 * NPRIMES
        kp = (K + 7) // 8 * 8
        n_pad = (N + 31) // 32 * 32
        # Algorithmic tensor FLOPs of one step's GEMM launches: each of the
        # `digits` digit planes of every (prime, part) plane is one d x k x n
        # product.  Rates divide each kernel's work per step by its summed
        # launch time per step.
        gemm_flops = 2.0 * D * K * N * planes * digits
        # Algorithmic bytes of a step's GEMMs: the f16 digit matrix read once,
        # U16 once per launch, the u64 outputs written once.
        gemm_per_step = max(gemm_n, 1) / args.steps
        gemm_bytes = (planes * K * digits * N * 2 + gemm_per_step * D * kp * 2 + planes * D * N * 8)
        gemm_step_s = gemm_ms / args.steps * 1e-3
        achieved = gemm_flops / gemm_step_s / 1e12
        peak, peak_kind = tensor_peak(peaks, elapsed_ms)
        split_bytes = planes * K * N * 8 + planes * (n_pad // 32) * digits * 32 * kp * 2
        split_gbs = split_bytes / (split_ms / args.steps * 1e-3) / 1e9

        # Decrypted result of the last timed step against the FP64 product U*M.
        dec = decrypt_error(U_np, M_np, sec, Aout, Bout, primes)
        ref_out = (Aout.view(torch.int64).clone(), Bout.view(torch.int64).clone())

        # FP64 comparison: cuBLAS DGEMM of U*M at the same n, and the FP64-limb path.
        Ud = U.to(torch.float64)
        Md = torch.from_numpy(np.ascontiguousarray(M_np)).to(dev)
        for _ in range(2):
            torch.matmul(Ud, Md)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        f0.record(stream)
        for _ in range(reps):
            torch.matmul(Ud, Md)
        f1.record(stream)
        torch.cuda.synchronize()
        dgemm_ms = f0.elapsed_time(f1) / reps
        del Ud, Md

        fp64_ms = None
        fp64_tight_ms = None
        fp64_identical = None
        fp64_roof = None
        if not args.no_fp64:
            pkg.pc_mm(U, A, B, primes, out=(Aout, Bout), path="fp64")
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            pkg.pc_mm(U, A, B, primes, out=(Aout, Bout), path="fp64")
            g1.record(stream)
            torch.cuda.synchronize()
            fp64_ms = g0.elapsed_time(g1)
            fp64_identical = bool(torch.equal(Aout.view(torch.int64), ref_out[0]) and
                                  torch.equal(Bout.view(torch.int64), ref_out[1]))
            # The tight asymmetric split: U is one digit (|U| <= 128), so A's base can be
            # 2^53 / (128 k), two digits per residue at k = 4096 instead of three.
            pkg.pc_mm(U, A, B, primes, out=(Aout, Bout), path="fp64_tight")
            torch.cuda.synchronize()
            g0.record(stream)
            pkg.pc_mm(U, A, B, primes, out=(Aout, Bout), path="fp64_tight")
            g1.record(stream)
            torch.cuda.synchronize()
            fp64_tight_ms = g0.elapsed_time(g1)
            fp64_identical = fp64_identical and bool(
                torch.equal(Aout.view(torch.int64), ref_out[0]) and
                torch.equal(Bout.view(torch.int64), ref_out[1]))
        del ref_out
        # The FP64-limb path against the FP64 peak: its DGEMMs (k1 * k2 per
        # (prime, part) plane, each 2*d*k*n FLOPs) over its time, divided by
        # the rate of the plain cuBLAS DGEMM measured above (the FP64 peak
        # this GPU delivers; the nominal dense FP64 rate is 1.25 TFLOP/s).
        dgemm_tflops = 2.0 * D * K * N / (dgemm_ms * 1e-3) / 1e12
        fp64_roof = {"peak": dgemm_tflops, "peak_source": "measured cuBLAS DGEMM U*M, same n",
                     "nominal_fp64_tflops": 1.25, "unit": "TFLOP/s"}
        for name, ms_, tight in (("paper_split", fp64_ms, False), ("tight_split", fp64_tight_ms, True)):
            if ms_ is None:
                continue
            info = pkg.plan_info(K, primes[0], "fp64_tight" if tight else "fp64")
            prods = info["digits"] * 1 * planes  # U is one base-K digit (|U| <= 128 < K)
            fl = 2.0 * D * K * N * prods
            fp64_roof[name] = {"dgemms": prods, "flops": fl,
                               "achieved": fl / (ms_ * 1e-3) / 1e12,
                               "frac": fl / (ms_ * 1e-3) / 1e12 / dgemm_tflops,
                               "exact_tops": mod_ops_per_step() / (ms_ * 1e-3) / 1e12}

        # End to end through the public call with host buffers: every step
        # copies its inputs in from pinned host memory, runs pc_mm and copies
        # its outputs back.  Steps are pipelined as a streaming user would:
        # three streams (copy in, compute, copy out) and two device buffer
        # sets, so step i's product overlaps step i+1's input copy and step
        # i-1's output copy.  The serial form (all three on one stream) is
        # reported beside it.
        U_h = torch.from_numpy(U_np).pin_memory()
        A_h = torch.from_numpy(A_np).pin_memory()
        B_h = torch.from_numpy(B_np).pin_memory()
        outs_h = [(torch.empty(Aout.shape, dtype=torch.uint64).pin_memory(),
                   torch.empty(Bout.shape, dtype=torch.uint64).pin_memory()) for _ in range(2)]
        dev_sets = [(U, A, B, Aout, Bout),
                    (torch.empty_like(U), torch.empty_like(A), torch.empty_like(B),
                     torch.empty_like(Aout), torch.empty_like(Bout))]
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_cmp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def e2e_step(i):
            b = i & 1
            Ud, Ad, Bd, Aod, Bod = dev_sets[b]
            Aoh, Boh = outs_h[b]
            s_in.wait_event(ev_cmp[b])           # buffer set b's last product has read it
            with torch.cuda.stream(s_in):
                Ud.copy_(U_h, non_blocking=True)
                Ad.copy_(A_h, non_blocking=True)
                Bd.copy_(B_h, non_blocking=True)
            ev_in[b].record(s_in)
            s_cmp.wait_event(ev_in[b])
            s_cmp.wait_event(ev_out[b])          # buffer set b's last outputs are copied out
            pkg.pc_mm(Ud, Ad, Bd, primes, out=(Aod, Bod), stream=s_cmp)
            ev_cmp[b].record(s_cmp)
            s_out.wait_event(ev_cmp[b])
            with torch.cuda.stream(s_out):
                Aoh.copy_(Aod, non_blocking=True)
                Boh.copy_(Bod, non_blocking=True)
            ev_out[b].record(s_out)

        e2e_steps = max(4, min(args.steps, 20))
        for i in range(2):
            e2e_step(i)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(s_in)
        for i in range(e2e_steps):
            e2e_step(i)
        s_out.wait_event(ev_cmp[(e2e_steps - 1) & 1])
        h1.record(s_out)
        torch.cuda.synchronize()
        e2e_ms = h0.elapsed_time(h1) / e2e_steps
        h2d = U_h.numel() + 8 * (A_h.numel() + B_h.numel())
        d2h = 8 * (outs_h[0][0].numel() + outs_h[0][1].numel())
        last = (e2e_steps - 1) & 1
        if not np.array_equal(outs_h[last][0][0, :4].numpy(), dev_sets[last][3][0, :4].cpu().numpy()):
            raise RuntimeError("e2e copy-back mismatch")

        def serial_step():
            U.copy_(U_h, non_blocking=True)
            A.copy_(A_h, non_blocking=True)
            B.copy_(B_h, non_blocking=True)
            pkg.pc_mm(U, A, B, primes, out=(Aout, Bout))
            outs_h[0][0].copy_(Aout, non_blocking=True)
            outs_h[0][1].copy_(Bout, non_blocking=True)

        serial_step()
        torch.cuda.synchronize()
        h0.record(stream)
        for _ in range(4):
            serial_step()
        h1.record(stream)
        torch.cuda.synchronize()
        e2e_serial_ms = h0.elapsed_time(h1) / 4

        cpu_tops, cpu_dt, cpu_rows, cpu_threads = oracle_rate(U_np, A_np, B_np, primes)

        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "d": D, "k": K, "N": N, "primes": NPRIMES,
                       "prime_bits": PRIME_BITS, "digits": digits, "path": "f16",
                       "l2": "inputs larger than L2 (805 MB of residues read per step)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"kernel": "gemm_f16_kernel", "bound": "tensor", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "peak_kind": peak_kind,
                         "peak_source": (f"{peak_src} bf16 dense {peak_kind} (f16 same rate); "
                                         f"burst for a timed region under 1 s "
                                         f"({elapsed_ms:.0f} ms here), sustained above"),
                         "frac_of_sustained": achieved / peaks["bf16_tflops_sustained"],
                         "traffic": GEMM_TRAFFIC_N4096 if (D, K, N) == (4096, 4096, 4096) else None,
                         "traffic_algorithmic": gemm_bytes / gemm_per_step,
                         "avg_launch_ms": gemm_step_s * 1e3 / gemm_per_step,
                         "flops_per_launch": gemm_flops / gemm_per_step,
                         "launches_per_step": gemm_per_step},
            "split_kernel": {"ms_per_step": split_ms / args.steps,
                             "launches_per_step": split_n / args.steps,
                             "achieved_gbs": split_gbs, "peak_gbs": peaks["hbm_gbs"],
                             "frac": split_gbs / peaks["hbm_gbs"]},
            "pc_mm_ms": ms_per_step,
            "fp64_matmul_ms": dgemm_ms,
            "slowdown_vs_fp64_matmul": ms_per_step / dgemm_ms,
            "fp64_limb_pc_mm_ms": fp64_ms,
            "fp64_limb_tight_pc_mm_ms": fp64_tight_ms,
            "fp64_limb_outputs_identical": fp64_identical,
            "fp64_limb_roofline": fp64_roof,
            "decrypt": dec,
            "int8_limb": "unavailable: tcgen05.mma kind::i8 is not supported on sm_103a (ptxas)",
            "cpu_baseline": {"value": cpu_tops, "unit": UNIT, "cores": cpu_threads,
                             "kind": "oracle",
                             "sample": f"{cpu_rows} of {D} output rows of all 6 planes, full k and n "
                                       f"({cpu_dt:.1f} s); rate extrapolated linearly"},
            "e2e": {"value": mod_ops_per_step() / (e2e_ms * 1e-3) / 1e12, "unit": UNIT,
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "pipelined": "copy-in, product and copy-out on three streams, two buffer sets",
                    "serial_ms_per_step": e2e_serial_ms,
                    "serial_value": mod_ops_per_step() / (e2e_serial_ms * 1e-3) / 1e12},
            "gpu_launches": (gemm_n + split_n + u16_n),
            "clocks": clk,
        }
        if not args.no_extra:
            # The rest of the metric, each with its own timed region after the
            # line's: the latency-bound 256^3 case, PC-MM at n=16384 and CC-MM
            # at n=8192.  The n=4096 buffers are released first.
            del dev_sets, U, A, B, Aout, Bout, U_h, A_h, B_h, outs_h
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            line["config1"] = measure_config1(pkg, dev, stream)
            line["strategy2"] = measure_strategy2(pkg, dev, stream, peaks)
            line["precomp"] = [measure_precomp(pkg, dev, stream, d3) for d3 in (4096, 32)]
            line["pcmm16384"] = measure_pc_large(pkg, dev, stream, "pcmm16384", 5, 3, peaks)
            line["ccmm"] = measure_ccmm(pkg, dev, stream, 8192, 5, 3, peaks, e2e=True,
                                        cpu_leg=False)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- secondary workloads
# Workloads measured beside the default PC-MM n=4096 line above.

def _timed(step, steps, warmup, stream, pkg):
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    pkg.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    kern = {name: pkg.profile_read(kid) for name, kid in
            (("gemm", pkg.KERNEL_GEMM), ("split", pkg.KERNEL_SPLIT), ("u16", pkg.KERNEL_U16))}
    pkg.profile_enable(False)
    return e0.elapsed_time(e1) / steps, kern


def measure_pc_large(pkg, dev, stream, workload: str, steps: int, warmup: int, peaks: dict):
    """PC-MM n=16384 (d = k = N = 16384, L = 4 primes of 50 bits) or PC-Mv
    (16384^2 int8 U times a batch of 32), inputs uniform on the device: time per
    step, exact TOPS, the GEMM's fraction of the tensor peak and, for PC-MM,
    the cuBLAS FP64 DGEMM of the same n and the slowdown against it."""
    import torch
    from paper_2503_16080_gb300 import synth
    d = k = 16384
    n = 16384 if workload == "pcmm16384" else 32
    P = 4
    primes = synth.ntt_primes(50, P)
    U = synth.uniform_int8_torch(SEED, 1, (d, k), dev)
    A = torch.stack([synth.uniform_mod_torch(SEED, 10 + j, (k, n), q, dev)
                     for j, q in enumerate(primes)])
    B = torch.stack([synth.uniform_mod_torch(SEED, 20 + j, (k, n), q, dev)
                     for j, q in enumerate(primes)])
    Ao = torch.empty((P, d, n), dtype=torch.uint64, device=dev)
    Bo = torch.empty_like(Ao)
    fn = pkg.pc_mm if workload == "pcmm16384" else pkg.pc_mv
    prepared = None
    if workload == "pcmv":
        # The plaintext reused over many products: converted to f16 once.
        prep = pkg.PreparedU(U)
        ms_p, kern_p = _timed(lambda: fn(prep, A, B, primes, out=(Ao, Bo)), steps, warmup, stream,
                              pkg)
        prepared = {"ms_per_step": ms_p, "tops": 2.0 * d * k * n * 2 * P / (ms_p * 1e-3) / 1e12,
                    "gemm_ms_per_step": kern_p["gemm"][0] / steps,
                    "note": "U converted once (PreparedU / pc_mm_u16), outside the timed steps"}
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    clocks.mark()
    ms, kern = _timed(lambda: fn(U, A, B, primes, out=(Ao, Bo)), steps, warmup, stream, pkg)
    clk = clocks.stop()
    ops = 2.0 * d * k * n * 2 * P
    L = pkg.plan_info(k, primes[0])["digits"]
    g_ms = kern["gemm"][0] / steps  # GEMM time per step (all launches of a step)
    gflops = ops * L
    peak, kind = tensor_peak(peaks, ms * steps)
    out = {
        "workload": workload, "value": ops / (ms * 1e-3) / 1e12, "ms_per_step": ms,
        "steps": steps, "warmup": warmup,
        "config": {"workload": (f"PC-MM n=16384: U 16384^2 int8 x 16384 row-RLWE cts of degree "
                                f"16384, L=4 primes of 50 bits" if n > 32 else
                                "PC-Mv: U 16384^2 int8 x batch of 32, L=4 primes of 50 bits"),
                   "d": d, "k": k, "n": n, "primes": P, "digits": L,
                   "digit_bits": pkg.get_digit_bits()},
        "roofline": {"kernel": "gemm_f16_kernel", "bound": "tensor",
                     "achieved": gflops / (g_ms * 1e-3) / 1e12, "peak": peak,
                     "peak_kind": kind, "unit": "TFLOP/s",
                     "frac": gflops / (g_ms * 1e-3) / 1e12 / peak,
                     "gemm_ms_per_step": g_ms,
                     "launches_per_step": kern["gemm"][1] / steps},
        "kernels_ms_per_step": {kname: v[0] / steps for kname, v in kern.items()},
        "hbm_gbs_U_stream": d * k * 2 / (g_ms * 1e-3) / 1e9,
        "prepared_u": prepared,
        "fp64_matmul_ms": None, "clocks": clk}
    del A, B, Ao, Bo
    if workload == "pcmm16384":
        Ud = U.to(torch.float64)
        del U
        Md = torch.empty((k, n), dtype=torch.float64, device=dev).uniform_(-1, 1)
        torch.matmul(Ud[:1024], Md)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        torch.matmul(Ud, Md)
        f1.record(stream)
        torch.cuda.synchronize()
        out["fp64_matmul_ms"] = f0.elapsed_time(f1)
        out["slowdown_vs_fp64_matmul"] = ms / out["fp64_matmul_ms"]
        del Ud, Md
    torch.cuda.empty_cache()
    return out


def measure_strategy2(pkg, dev, stream, peaks: dict, steps: int = 5, warmup: int = 3):
    """Strategy 2 of Sec. 6.1 (truncation) in the paper's single-modulus
    setting: one 54-bit modulus, d = k = n = 4096, U the benchmark's int8
    plaintext, B uniform residues (an RLWE b-part is indistinguishable from
    uniform).  Times the exact product (f16 digits), the f16 truncation with
    s = 9 and 18 dropped bits (one and two fewer digit products) and the
    binary64 form as printed (one DGEMM); reports each result's largest
    centred deviation from the exact product against its bound."""
    import torch
    from paper_2503_16080_gb300 import synth
    n = 4096
    q = synth.ntt_primes(54, 1)[0]
    U = torch.from_numpy(synth.quantised_normal_int8(SEED, 1, (n, n))).to(dev)
    B = synth.uniform_mod_torch(SEED, 40, (n, n), q, dev)
    exact = torch.empty((n, n), dtype=torch.uint64, device=dev)
    out = torch.empty_like(exact)
    normU = int(U.abs().max())
    normB = (q - 1) // 2
    res = {"workload": "one modulus q ~ 2^54 (54-bit prime), d = k = n = 4096, U int8 "
                       "(N(0,1)*2^5), B uniform mod q", "q_bits": q.bit_length(), "forms": []}
    ops = 2.0 * n ** 3
    forms = [("f16 exact", "f16", 0), ("f16 trunc s=9", "f16", 9), ("f16 trunc s=18", "f16", 18),
             ("fp64 as printed", "fp64", 0)]
    for name, path, sbits in forms:
        dst = exact if name == "f16 exact" else out
        ms, kern = _timed(lambda: pkg.modpp_mm_trunc(U, B, q, path=path, drop_bits=sbits, out=dst),
                          steps if path == "f16" else 2, warmup if path == "f16" else 1, stream, pkg)
        row = {"form": name, "ms": ms, "tops": ops / (ms * 1e-3) / 1e12}
        if path == "f16":
            wsb = int(pkg.lib().modpp_mm_trunc_workspace(n, n, n, q, 0, sbits))
            row["gemm_ms"] = kern["gemm"][0] / max(kern["gemm"][1], 1)
            row["workspace_bytes"] = wsb
            row["bound"] = n * normU * 2 ** (sbits - 1) if sbits else 0
        else:
            row["bound"] = 2.0 ** -50 * n * normU * normB
            row["fp64_tflops"] = ops / (ms * 1e-3) / 1e12
        if name != "f16 exact":
            d = (out.view(torch.int64) - exact.view(torch.int64))
            d = torch.remainder(d, q)
            d = torch.where(d > q // 2, d - q, d)
            row["max_abs_err"] = int(d.abs().max())
            row["within_bound"] = row["max_abs_err"] <= row["bound"]
            row["err_over_scale_2^45"] = row["max_abs_err"] / 2.0 ** 45
        res["forms"].append(row)
    del U, B, exact, out
    torch.cuda.empty_cache()
    return res


def measure_precomp(pkg, dev, stream, d3: int, steps: int = 5, warmup: int = 3):
    """Alg. 7 (CP-MM with precomputation) with the key switches back to one
    secret, against Alg. 6 (pc_mm, two Mod-PP-MMs) on the same shape: ring
    degree N = d2 = 4096, d3 output columns, L = 3 primes of 50 bits and a
    60-bit special prime.  Inputs uniform mod q (RLWE parts and keys are
    indistinguishable from uniform; the kernels' work does not depend on the
    values)."""
    import torch
    from paper_2503_16080_gb300 import synth
    N = d2 = 4096
    L = 3
    primes = synth.ntt_primes(50, L)
    prp = primes + synth.ntt_primes(60, 1)
    ring = pkg.Ring(N, prp)
    Ut = torch.from_numpy(synth.quantised_normal_int8(SEED, 1, (d3, d2))).to(dev)
    a = torch.stack([synth.uniform_mod_torch(SEED, 50 + j, (N,), q, dev) for j, q in enumerate(primes)])
    B = torch.stack([synth.uniform_mod_torch(SEED, 60 + j, (d2, N), q, dev)
                     for j, q in enumerate(primes)])
    keys = torch.empty((d3,) + ring.key_shape(), dtype=torch.uint64, device=dev)
    kv = keys.view(torch.int64)
    for k, q in enumerate(prp):
        kv[:, :, :, k, :] = synth.uniform_mod_torch(SEED, 70 + k, (d3, L, 2, N), q,
                                                    dev).view(torch.int64)
    ring.prepare_keys(keys)
    out = torch.empty((2, L, d3, N), dtype=torch.uint64, device=dev)
    ws = torch.empty(int(pkg.lib().pc_mm_precomp_workspace(ring._h, d2, d3, 0)), dtype=torch.uint8,
                     device=dev)
    ms7, kern = _timed(lambda: ring.pc_mm_precomp(Ut, a, B, keys, out=out, workspace=ws),
                       steps, warmup, stream, pkg)
    gemm7 = kern["gemm"][0] / steps
    # Alg. 6 on the same shape: both parts (a-parts A and b-parts B) times U^T.
    A = torch.stack([synth.uniform_mod_torch(SEED, 80 + j, (d2, N), q, dev)
                     for j, q in enumerate(primes)])
    Ao = torch.empty((L, d3, N), dtype=torch.uint64, device=dev)
    Bo = torch.empty_like(Ao)
    ms6, kern6 = _timed(lambda: pkg.pc_mm(Ut, A, B, primes, out=(Ao, Bo)), steps, warmup,
                        stream, pkg)
    res = {"workload": f"Alg. 7 with key switches vs Alg. 6: N = d2 = 4096, d3 = {d3}, L = 3 "
                       "(50-bit) + 60-bit special prime, U int8",
           "d2": d2, "d3": d3, "N": N,
           "alg7_ms": ms7, "alg7_gemm_ms": gemm7, "alg7_keyswitch_ms": ms7 - gemm7
           - kern["split"][0] / steps - kern["u16"][0] / steps,
           "alg6_pc_mm_ms": ms6, "alg6_gemm_ms": kern6["gemm"][0] / steps,
           "mod_ops": 2.0 * d3 * d2 * N * L,
           "alg7_exact_tops_of_product": 2.0 * d3 * d2 * N * L / (gemm7 * 1e-3) / 1e12,
           "key_bytes": keys.numel() * 8}
    ring.close()
    del keys, A, B, out, ws, Ao, Bo
    torch.cuda.empty_cache()
    return res


def measure_config1(pkg, dev, stream, calls: int = 200):
    """The 256^3 Mod-PP-MM with one 50-bit prime and int32 U (values in
    [-128, 127]): the latency-bound case.  Reports the device time per call
    of back-to-back calls (CUDA events), the time of one call followed by a
    synchronisation (median), and the host time spent enqueueing one call."""
    import numpy as np
    import torch
    from paper_2503_16080_gb300 import synth
    n = 256
    q = synth.ntt_primes(50, 1)
    U = torch.from_numpy(synth.uniform_int8(1, 1, (n, n)).astype(np.int32)).to(dev)
    A = synth.uniform_mod_torch(1, 2, (1, n, n), q[0], dev)
    C = torch.empty((1, n, n), dtype=torch.uint64, device=dev)
    ws = torch.empty(pkg.workspace_bytes(n, n, n, q), dtype=torch.uint8, device=dev)

    def call():
        pkg.modpp_mm(U, A, q, out=C, workspace=ws)

    for _ in range(20):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    for _ in range(calls):
        call()
    t_enq = time.perf_counter() - t0
    e1.record(stream)
    torch.cuda.synchronize()
    back_to_back = e0.elapsed_time(e1) / calls
    sync = []
    for _ in range(50):
        t0 = time.perf_counter()
        call()
        torch.cuda.synchronize()
        sync.append(time.perf_counter() - t0)
    pkg.profile_enable(True)
    call()
    launches = sum(pkg.profile_read(kid)[1]
                   for kid in (pkg.KERNEL_GEMM, pkg.KERNEL_SPLIT, pkg.KERNEL_U16))
    pkg.profile_enable(False)
    return {"workload": "Mod-PP-MM 256^3, one 50-bit prime, int32 U in [-128,127] "
                        "(uniform), A uniform mod q",
            "d": n, "k": n, "n": n, "primes": 1,
            "us_per_call_back_to_back": back_to_back * 1e3,
            "us_per_call_with_sync": statistics.median(sync) * 1e6,
            "host_enqueue_us_per_call": t_enq / calls * 1e6,
            "launches_per_call": launches,
            "tops_back_to_back": 2.0 * n ** 3 / (back_to_back * 1e-3) / 1e12}


def run_secondary(args):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16080_gb300 as pkg
    from paper_2503_16080_gb300 import synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    if args.digit_bits:
        pkg.set_digit_bits(args.digit_bits)
    peaks, peak_src = load_peaks()
    clocks = ClockSampler(0)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16", "data": "synthetic"}
    if args.workload in ("pcmm16384", "pcmv"):
        line.update(measure_pc_large(pkg, dev, stream, args.workload, args.steps, args.warmup,
                                     peaks))
    elif args.workload == "strategy2":
        line.update({"workload": "strategy2", **measure_strategy2(pkg, dev, stream, peaks,
                                                                  args.steps, args.warmup)})
    elif args.workload == "precomp":
        line.update({"workload": "precomp",
                     "rows": [measure_precomp(pkg, dev, stream, d3, args.steps, args.warmup)
                              for d3 in (4096, 256, 32)]})
    elif args.workload == "hostlink":
        # Pinned host <-> device copy rates (the bound of the end-to-end
        # numbers): one direction at a time, and both at once on separate
        # streams; 400 MB per copy, CUDA events around each timed batch.
        nbytes = 400 << 20
        hb = [torch.empty(nbytes // 8, dtype=torch.int64).pin_memory() for _ in range(2)]
        db = [torch.empty(nbytes // 8, dtype=torch.int64, device=dev) for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def rate(copies, reps=5):
            for _ in range(2):
                copies()
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                s_in.wait_stream(stream)
                s_out.wait_stream(stream)
                copies()
                stream.wait_stream(s_in)
                stream.wait_stream(s_out)
            t1.record(stream)
            torch.cuda.synchronize()
            return t0.elapsed_time(t1) / reps

        def h2d():
            with torch.cuda.stream(s_in):
                db[0].copy_(hb[0], non_blocking=True)

        def d2h():
            with torch.cuda.stream(s_out):
                hb[1].copy_(db[1], non_blocking=True)

        def both():
            h2d()
            d2h()

        ms_in, ms_out, ms_both = rate(h2d), rate(d2h), rate(both)
        step_in, step_out = 822083584, 805306368  # bytes per PC-MM n=4096 step (e2e)
        bidir = 2 * nbytes / (ms_both * 1e-3) / 1e9
        line.update({"workload": "hostlink", "unit": "GB/s", "value": bidir,
                     "config": {"workload": "pinned host <-> device copies, 400 MB each"},
                     "h2d_gbs": nbytes / (ms_in * 1e-3) / 1e9,
                     "d2h_gbs": nbytes / (ms_out * 1e-3) / 1e9,
                     "bidirectional_gbs": bidir,
                     "pcmm4096_e2e_bound_ms": (step_in + step_out) / (bidir * 1e9) * 1e3})
    elif args.workload == "umma_sweep":
        # Tensor throughput of the digit GEMM against UMMA N: one plane of
        # 8192^3 with primes of 9, 18, 27, 36, 45 and 50 bits gives L = 1..6
        # digits of 9 bits and tile widths N = L * tile_cols(L).
        d = k = n = 8192
        U = synth.uniform_int8_torch(SEED, 1, (d, k), dev)
        rows = []
        for bits in (9, 18, 27, 36, 45, 50):
            q = synth.ntt_primes(bits, 1, two_adicity=1)[0]
            A = synth.uniform_mod_torch(SEED, 2, (1, k, n), q, dev)
            C = torch.empty((1, d, n), dtype=torch.uint64, device=dev)
            ms, kern = _timed(lambda: pkg.modpp_mm(U, A, [q], out=C), args.steps, args.warmup,
                              stream, pkg)
            L = pkg.plan_info(k, q)["digits"]
            g_ms = kern["gemm"][0] / args.steps
            tf = 2.0 * d * k * n * L / (g_ms * 1e-3) / 1e12
            rows.append({"prime_bits": bits, "digits": L, "umma_n": L * {1: 64, 2: 64, 3: 64,
                                                                         4: 48, 5: 48, 6: 40}[L],
                         "gemm_ms": g_ms, "tflops": tf,
                         "frac": tf / peaks["bf16_tflops_sustained"]})
        line.update({"workload": "umma_sweep", "unit": "TFLOP/s", "value": rows[-1]["tflops"],
                     "config": {"workload": "digit GEMM, one plane of 8192^3, L = 1..6 digits"},
                     "rows": rows})
    elif args.workload == "grouped":
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        seed = 3
        w = synth.u64(seed, 1, 4 * 64)
        probs = []
        ops = 0.0
        for i in range(64):
            dd, kk, nn = (256 << int(w[4 * i + j] % np.uint64(6)) for j in range(3))
            P = 1 + int(w[4 * i + 3] % np.uint64(6))
            primes = synth.random_primes(seed, 1000 + i, P, 40, 60)
            U = synth.uniform_int8_torch(seed, 2000 + i, (dd, kk), dev)
            A = torch.stack([synth.uniform_mod_torch(seed, 10000 + 16 * i + j, (kk, nn), q, dev)
                             for j, q in enumerate(primes)])
            probs.append((U, A, primes))
            ops += 2.0 * dd * kk * nn * P
        plan = pkg.GroupedPlan(probs, tune=True)
        clocks.start()
        ms_graph, _ = _timed(lambda: plan.run(graph=True), args.steps, args.warmup, stream, pkg)
        clk = clocks.stop()
        # Per-kernel times of the same launches without the graph (events
        # are not recorded inside a replayed graph).
        ms_direct, kern = _timed(lambda: plan.run(graph=False), args.steps, args.warmup, stream,
                                 pkg)
        outs = [torch.empty_like(C) for C in plan.outputs]

        def per_problem():
            for (U, A, primes), C in zip(probs, outs):
                pkg.modpp_mm(U, A, primes, out=C)

        pkg.set_digit_bits(plan.info()["digit_bits"])
        ms_loop, kern_loop = _timed(per_problem, args.steps, args.warmup, stream, pkg)
        same = all(torch.equal(a, b) for a, b in zip(plan.outputs, outs))
        line.update({
            "workload": "grouped", "value": ops / (ms_graph * 1e-3) / 1e12, "ms_per_step": ms_graph,
            "config": {"workload": "64 uneven Mod-PP-MMs: d,k,n in 256*2^{0..5}, 1-6 primes of "
                                   "40-60 bits, one grouped plan replayed as a CUDA graph",
                       "problems": 64, "mod_ops": ops, "plan": plan.info()},
            "per_problem_launches_ms": ms_loop,
            "grouped_speedup": ms_loop / ms_graph,
            "grouped_equals_per_problem": same,
            "launches_grouped": 3, "launches_per_problem": 3 * 64,
            "plan_direct_ms": ms_direct,
            "kernels_ms_per_step_grouped": {kname: v[0] / args.steps for kname, v in kern.items()},
            "kernels_ms_per_step_per_problem": {kname: v[0] / args.steps
                                                for kname, v in kern_loop.items()},
            "clocks": clk})
        plan.close()
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- CC-MM

CC_WORKLOAD = ("CC-MM n=8192 (Alg. 8): two column-wise encrypted 8192x8192 matrices, ring degree "
               "8192, L=4 primes of 50 bits, key switching with {gadget}, N automorphism keys "
               "and a relinearisation key resident on the device; output rescaled by q_3; real "
               "encryptions of M1, M2 uniform in [-1,1] at scale 2^40 under a ternary secret")
# Key-switching gadgets of the CC-MM workload: the paper's experimental
# setting (Sec. 6: dnum = 2), two digits of two chain primes over two 60-bit
# special primes; and one digit per chain prime over one special prime.
CC_GADGETS = {"paper": (2, 2, "dnum=2 digits of two primes + two 60-bit special primes "
                                "(the paper's dnum)"),
              "prime": (None, 1, "dnum=L one-prime digits + one 60-bit special prime")}


def measure_ccmm(pkg, dev, stream, Nr: int, steps: int, warmup: int, peaks: dict,
                 e2e: bool = True, cpu_leg: bool = True, gadget: str = "paper"):
    """CC-MM (Alg. 8) at ring degree Nr, L = 4, with the key-switching gadget
    CC_GADGETS[gadget]: harness (real encryptions and keys), timed steps,
    stage split, CRT GEMM roofline, FP64 DGEMM of the same n, decrypted error;
    optionally the end-to-end form from host memory and the CPU oracle's
    extrapolated time.  Returns the measurement as a dict."""
    import numpy as np
    import torch
    from paper_2503_16080_gb300 import synth

    L = 4
    dnum, K, gadget_text = CC_GADGETS[gadget]
    dnum = L if dnum is None else dnum
    primes = synth.ntt_primes(50, L)
    prp = primes + synth.ntt_primes(60, K)
    ring = pkg.Ring(Nr, prp, special=K, dnum=dnum)

    # Real inputs: column-wise encryptions of M1 and M2 under a ternary secret,
    # valid automorphism and relinearisation keys (the kernels' work does not
    # depend on the values; the decrypted product is checked after timing).
    t_h = time.perf_counter()
    inp = ccmm_inputs(Nr, primes, prp, dev, dnum=dnum)
    torch.cuda.synchronize()
    harness_s = time.perf_counter() - t_h
    ct1, ct2 = inp["ct1"], inp["ct2"]
    t_k = time.perf_counter()
    keys = ring.prepare_keys(inp["keys"])   # in place: evaluation-domain Montgomery form
    rkey = ring.prepare_keys(inp["rkey"])
    torch.cuda.synchronize()
    prepare_s = time.perf_counter() - t_k
    out = torch.empty((2, L - 1, Nr, Nr), dtype=torch.uint64, device=dev)
    ws_bytes = ring.cc_mm_workspace_bytes()
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)

    def step():
        ring.cc_mm(ct1, ct2, keys, rkey, out=out, workspace=ws)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    region_ms = e0.elapsed_time(e1)
    ms = region_ms / steps
    dec = ccmm_decrypt_error(inp, out, primes)

    # Stage split and GEMM launches (one extra, separately timed call).
    pkg.profile_enable(True)
    step()
    stages = ring.cc_mm_stage_ms()
    gemm_ms, gemm_n = pkg.profile_read(pkg.KERNEL_GEMM)
    pre_ms, pre_n = pkg.profile_read(pkg.KERNEL_SPLIT)
    post_ms, post_n = pkg.profile_read(pkg.KERNEL_U16)
    pkg.profile_enable(False)

    crt_primes = pkg.wide_plan_info(Nr, primes)
    if crt_primes:
        # CRT form: R small-prime products of [A;B] (2N x N) times an N x N
        # operand per (chain prime, right operand), over pieces of k.
        products = crt_primes
        form = {"form": "crt", "small_primes": crt_primes}
    else:
        LU = -(-(max(primes) - 1).bit_length() // 8)
        LA = pkg.plan_info(Nr, primes[0])["digits"]
        products = LU * LA
        form = {"form": "digits", "u_digit_planes": LU, "a_digits": LA}
    # Tensor work of all GEMM launches of one CC-MM: 2 right operands x L
    # chain primes x `products` products of 2N x N x N.
    total_flops = 2.0 * (2 * Nr) * Nr * Nr * products * 2 * L
    gemm_flops = total_flops / max(gemm_n, 1)
    g_avg = gemm_ms / max(gemm_n, 1)
    achieved = total_flops / (gemm_ms * 1e-3) / 1e12
    peak, kind = tensor_peak(peaks, region_ms)
    modops = 2.0 * (2 * Nr) * Nr * (2 * Nr) * L

    # FP64 matmul of the same n.
    Ad = torch.empty((Nr, Nr), dtype=torch.float64, device=dev).uniform_(-1, 1)
    Bd = torch.empty_like(Ad).uniform_(-1, 1)
    torch.matmul(Ad, Bd)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    torch.matmul(Ad, Bd)
    f1.record(stream)
    torch.cuda.synchronize()
    dgemm_ms = f0.elapsed_time(f1)
    del Ad, Bd

    e2e_out = None
    if e2e:
        # End to end: both ciphertext matrices from pinned host memory, the
        # product, and the result back, every step (keys stay resident).
        h1 = torch.empty(ct1.shape, dtype=torch.uint64).pin_memory()
        h2 = torch.empty(ct2.shape, dtype=torch.uint64).pin_memory()
        ho = torch.empty(out.shape, dtype=torch.uint64).pin_memory()
        h1.copy_(ct1)
        h2.copy_(ct2)
        marks = []

        def e2e_step(record=False):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)] if record else None
            ct1.copy_(h1, non_blocking=True)
            ct2.copy_(h2, non_blocking=True)
            if record:
                ev[0].record(stream)
            step()
            if record:
                ev[1].record(stream)
            ho.copy_(out, non_blocking=True)
            if record:
                ev[2].record(stream)
                marks.append(ev)

        e2e_step()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_steps = max(1, min(steps, 3))
        g0.record(stream)
        for _ in range(e2e_steps):
            e2e_step(record=True)
        g1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = g0.elapsed_time(g1) / e2e_steps
        # Per part: copy-in (from the previous step's end), product, copy-out.
        starts = [g0] + [m[2] for m in marks[:-1]]
        e2e_out = {"value": e2e_ms, "unit": "ms per CC-MM",
                   "h2d_bytes_per_step": 8 * (h1.numel() + h2.numel()),
                   "d2h_bytes_per_step": 8 * ho.numel(),
                   "parts": {
                       "h2d_ms": sum(a.elapsed_time(m[0]) for a, m in zip(starts, marks)) / e2e_steps,
                       "cc_mm_ms": sum(m[0].elapsed_time(m[1]) for m in marks) / e2e_steps,
                       "d2h_ms": sum(m[1].elapsed_time(m[2]) for m in marks) / e2e_steps}}

    # CPU oracle on a small ring (N=512): the whole CC-MM, and its Mod-PP-MM
    # part alone; the products extrapolate by N^3, the rest (transposes, key
    # switches, relin) by N^2 log N.
    cpu = None
    if cpu_leg:
        import oracle
        oracle.build()
        n0 = 512
        kz = [None] + [np.zeros((dnum, 2, L + K, n0), dtype=np.uint64)] * (n0 - 1)
        c0 = np.zeros((n0, 2, L, n0), dtype=np.uint64)
        for j, q in enumerate(primes):
            c0[:, :, j, :] = synth.uniform_mod(SEED, 700 + j, (n0, 2, n0), q)
        t0 = time.perf_counter()
        oracle.cc_mm(c0, c0, kz, np.zeros((dnum, 2, L + K, n0), dtype=np.uint64), prp)
        t_all = time.perf_counter() - t0
        Ub = np.concatenate([c0[:, 0, 0, :].T, c0[:, 1, 0, :].T])
        Wb = np.concatenate([c0[:, 0, 0, :], c0[:, 1, 0, :]], axis=1)
        t0 = time.perf_counter()
        oracle.mod_pp_mm_residues(Ub, Wb, primes[0])
        t_mm = (time.perf_counter() - t0) * L
        f = Nr / n0
        est = t_mm * f ** 3 + max(t_all - t_mm, 0.0) * f ** 2 * np.log2(Nr) / np.log2(n0)
        cpu = {"value": est * 1e3, "unit": "ms per CC-MM",
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
               "kind": "oracle",
               "sample": f"one oracle CC-MM at N={n0} ({t_all:.1f} s, of which {t_mm:.1f} s in the "
                         f"step-2 products); products scaled by (N/{n0})^3, the rest by "
                         f"(N/{n0})^2 log N"}

    res = {"workload": "ccmm8192" if Nr == 8192 else f"ccmm{Nr}",
           "value": ms, "unit": "ms per CC-MM", "higher_is_better": False,
           "steps": steps, "warmup": warmup, "ms_per_step": ms,
           "dtype": "u64 residues (f16 digits on tcgen05)",
           "config": {"workload": CC_WORKLOAD.format(gadget=gadget_text).replace("8192", str(Nr)),
                      "N": Nr, "L": L, "dnum": dnum, "special_primes": K,
                      "prime_bits": 50, "special_prime_bits": 60,
                      "l2": "inputs larger than L2", "key_bytes": keys.numel() * 8,
                      "workspace_bytes": ws_bytes},
           "stages_ms": {"transpose_ct2": stages[0], "mod_pp_mm_x2": stages[1],
                         "transpose_C00_C10": stages[2], "relin_finish": stages[3]},
           "mod_pp_mm_tops": modops / (stages[1] * 1e-3) / 1e12,
           "roofline": {"kernel": "gemm_f16_kernel", "bound": "tensor", "achieved": achieved,
                        "peak": peak, "peak_kind": kind, "unit": "TFLOP/s",
                        "frac": achieved / peak,
                        "frac_of_sustained": achieved / peaks["bf16_tflops_sustained"],
                        "avg_launch_ms": g_avg, "launches_per_cc_mm": gemm_n,
                        "flops_per_launch": gemm_flops, "flops_per_cc_mm": total_flops, **form},
           "wide_passes_ms": {"gemm": gemm_ms, "residue_split": pre_ms, "crt_or_u16": post_ms},
           "fp64_matmul_ms": dgemm_ms, "slowdown_vs_fp64_matmul": ms / dgemm_ms,
           "decrypt": dec,
           "harness_s": {"encrypt_and_keygen": harness_s, "prepare_keys": prepare_s,
                         "note": "not in the timed region"},
           "e2e": e2e_out, "cpu_baseline": cpu, "clocks": clk}
    ring.close()
    del inp, keys, rkey, ct1, ct2, out, ws
    torch.cuda.empty_cache()
    return res


def run_ccmm(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16080_gb300 as pkg

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    peaks, _ = load_peaks()
    res = measure_ccmm(pkg, dev, stream, args.ccmm_n, args.steps, args.warmup, peaks,
                       gadget=args.gadget,
                       e2e=True, cpu_leg=not args.quick)
    line = {"metric": METRIC, **res, "n_gpus": 1, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic"}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-limb comparison")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload: skip the config-1, n=16384 and CC-MM sub-objects")
    ap.add_argument("--quick", action="store_true",
                    help="timed loop only (no FP64, e2e or CPU legs): for profiler runs")
    ap.add_argument("--digit-bits", type=int, default=0,
                    help="digit width of the f16 path (8, 9, 10; 0 = library default)")
    ap.add_argument("--workload", default="pcmm4096",
                    choices=["pcmm4096", "pcmm16384", "pcmv", "grouped", "ccmm8192",
                             "umma_sweep", "hostlink", "strategy2", "precomp"],
                    help="pcmm4096 (default, the benchmark line); the others are recorded "
                         "beside it")
    ap.add_argument("--n", type=int, default=4096,
                    help="square size d = k = N (default 4096, the benchmark workload)")
    ap.add_argument("--gadget", default="paper", choices=sorted(CC_GADGETS),
                    help="key-switching gadget of the ccmm8192 workload: paper (dnum=2, two "
                         "special primes) or prime (one digit per chain prime, one special)")
    ap.add_argument("--ccmm-n", type=int, default=8192,
                    help="ring degree of the ccmm8192 workload (smaller for profiling)")
    args = ap.parse_args()
    global D, K, N, WORKLOAD
    if args.n != 4096:
        D = K = N = args.n
        WORKLOAD = WORKLOAD.replace("n=4096", f"n={args.n}").replace("4096", str(args.n))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ccmm8192":
        return run_ccmm(args)
    if args.workload != "pcmm4096":
        return run_secondary(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
