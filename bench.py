#!/usr/bin/env python
"""Benchmark of the vertical secure-XGBoost Paillier hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config level] [--impl ours|reference]

One step is one pass of the whole hot path over one batch of synthetic input
(Sec. III.B's vertical pattern at Sec. III.C's worked scale):
  encode g/h -> encrypt (2M values) -> Montgomery form at the passive party ->
  encrypted histogram of every node of the level -> CRT decrypt of every cell ->
  decode.
Inputs are resident in HBM when the timed region starts; a second timed loop
(`e2e`) goes through the same public API from pinned host buffers, with the
host->device copies of the step's inputs and the device->host copy of the
decoded histogram inside the timed region.

Prints ONE JSON line on rank 0.  Under torchrun (N > 1) every rank runs an
independent replica of the workload (the path shards by sample and feature
with no exchange; weak scaling) and the slowest rank's time is used.

--impl reference runs the CPU oracle (plain Python integers) on a bounded
sample of the same workload on the host cores, rank 0 only.
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

from paper_2504_03909_b300 import synth  # noqa: E402

METRIC = "2048-bit Paillier enc/s & encrypted-hist ct-mults/s; p50/p99 request ms"

# DRAM bytes (read + write) per encryption of the current encryption kernel that dominates the
# step (the second stage when encryption runs as two launches), from an ncu capture of
# 16,384 encryptions of this kernel version, keyed by (n_bits, window)
TRAFFIC_PER_ENC = {(2048, 6): (164.205568e6 + 241.173760e6) / 16384}


# ----------------------------------------------------------------------------
# algorithmic work (integer multiply-add halves; a 32x32->64 limb product = 2)

def mont_imad(nl: int) -> int:
    """One CIOS Montgomery product on nl limbs: 2 nl^2 limb products + nl mul.lo."""
    return 4 * nl * nl + nl


def sliding_ops(e: int, w: int) -> int:
    """Length of the left-to-right sliding-window schedule of exponent e > 0 as
    the kernel runs it: one op for the leading window, then per zero bit outside
    a window one squaring, per window of len bits len squarings + one product."""
    i, n = e.bit_length() - 1, 0
    while i >= 0:
        if not (e >> i) & 1:
            n, i = n + 1, i - 1
            continue
        j = max(i - w + 1, 0)
        while not (e >> j) & 1:
            j += 1
        n += 1 if n == 0 else (i - j + 1) + 1
        i = j - 1
    return n


def exp_montmuls(e: int, w: int, pre: int = 2, post: int = 1) -> int:
    """Montgomery products of one exponentiation: `pre` to enter Montgomery form,
    the odd-power table (one squaring + 2^(w-1) - 1 products), the schedule after
    its leading window, `post` to leave."""
    return pre + (1 << (w - 1)) + (sliding_ops(e, w) - 1) + post


def schedule_split(e: int, w: int):
    """(squarings, products) of the sliding-window schedule after its leading window."""
    i, sq, pr, first = e.bit_length() - 1, 0, 0, True
    while i >= 0:
        if not (e >> i) & 1:
            sq, i = sq + 1, i - 1
            continue
        j = max(i - w + 1, 0)
        while not (e >> j) & 1:
            j += 1
        if first:
            first = False
        else:
            sq, pr = sq + (i - j + 1), pr + 1
        i = j - 1
    return sq, pr


def sos_shape(nl: int, lanes: int) -> bool:
    """Whether the exponentiation kernel at nl limbs and `lanes` lanes runs its
    schedule through the separated-form body (a multiple of 4 limbs per lane, at
    most 24, 4 to 16 lanes)."""
    s = nl // lanes
    return nl % lanes == 0 and s % 4 == 0 and 4 <= s <= 24 and 4 <= lanes <= 16 and lanes & (lanes - 1) == 0


def sos_square_imad(nl: int, lanes: int) -> int:
    """One separated-form squaring on nl limbs over `lanes` lanes of s limbs:
    per lane (lanes/2 - 1) s^2 limb products in the pair rounds, s^2/2 in the
    half round and s^2 in the diagonal round, then the reduction rows (nl^2 limb
    products + nl mul.lo over the instance).  A product through the same body
    forms lanes s^2 per lane: mont_imad(nl), as CIOS."""
    s = nl // lanes
    per_lane = (lanes // 2 - 1) * s * s + s * s // 2 + s * s
    return 2 * lanes * per_lane + 2 * nl * nl + nl


def exp_imad(e: int, w: int, nl: int, lanes: int, pre: int = 2, post: int = 1) -> int:
    """Multiply-add halves one exponentiation executes: CIOS products to enter
    Montgomery form, for the odd-power table and to leave it; the schedule's
    squarings and products through the separated-form body where the shape has
    it (else CIOS)."""
    sq, pr = schedule_split(e, w)
    cios = (pre + (1 << (w - 1)) + post) * mont_imad(nl)
    if sos_shape(nl, lanes):
        return cios + sq * sos_square_imad(nl, lanes) + pr * mont_imad(nl)
    return cios + (sq + pr) * mont_imad(nl)


def enc_split(L: int, lanes: int) -> bool:
    """Whether encryption runs as two launches (first stage at half the lanes)."""
    return (L, lanes) in ((64, 4), (96, 8))


def enc_imad_stages(n_bits: int, w: int, p: int, q: int, lanes: int = 4, cios: bool = False):
    """One encryption as the kernels run it, per CRT half (prime x, other prime
    x'): first stage mod x (L/2 limbs) with exponent x' mod (x - 1), second stage
    mod x^2 (L limbs) with exponent x; `lanes` is the second stage's lane count
    (the first stage runs at half of it when split, else at the same).  cios:
    every product counted at the CIOS cost (the count before squarings formed
    cross products once).  Returns (first, second)."""
    L = n_bits // 32
    if cios:
        first = sum(exp_montmuls(xo % (x - 1), w) for x, xo in ((p, q), (q, p))) * mont_imad(L // 2)
        second = sum(exp_montmuls(x, w) for x in (p, q)) * mont_imad(L)
        return first, second
    l1 = lanes // 2 if enc_split(L, lanes) else lanes
    first = sum(exp_imad(xo % (x - 1), w, L // 2, l1) for x, xo in ((p, q), (q, p)))
    second = sum(exp_imad(x, w, L, lanes) for x in (p, q))
    return first, second


def enc_imad(n_bits: int, w: int, p: int, q: int, lanes: int = 4, cios: bool = False) -> int:
    return sum(enc_imad_stages(n_bits, w, p, q, lanes, cios))


def dec_imad(n_bits: int, w: int, p: int | None = None, q: int | None = None, lanes: int | None = None) -> int:
    """One CRT decryption: c^(x - 1) mod x^2 per half.  Without the primes, an
    exponent of n_bits/2 bits with half its bits set stands in; without lanes,
    every product at the CIOS cost."""
    L = n_bits // 32
    es = [int("10" * (n_bits // 4), 2)] * 2 if p is None else [p - 1, q - 1]
    if lanes is None:
        return sum(exp_montmuls(e, w) for e in es) * mont_imad(L)
    return sum(exp_imad(e, w, L, lanes) for e in es)


# ----------------------------------------------------------------------------

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


IMAD_LANES_PER_SM = 64  # 4 SM sub-partitions x 16 lanes of the integer multiply-add pipe per clock
MAX_SM_MHZ = 2032.0     # B300 maximum SM clock
FP64_NOMINAL_TFLOPS = 1.25


def imad_peak_derived(sms: int) -> float:
    """The integer multiply-add roof in IMAD/s (1 IMAD = one 32-bit half of a
    32x32 -> 64 limb product): SMs x 64 lanes/clk x the maximum SM clock."""
    return sms * IMAD_LANES_PER_SM * MAX_SM_MHZ * 1e6


def plaintext_root_sums(P, torch, v, bins_d, M: int, F: int, K: int):
    """Untimed check data: per (feature, bin) of the root, the plain sums of the
    encoded g and h values and the sample counts (torch index_add / bincount on
    the device).  Every ciphertext enters F cells of the root histogram, so a
    decrypted root equal to these sums checks every ciphertext of the step
    through the homomorphism."""
    m = P.encode(v)
    idx = (torch.arange(F, device=v.device)[:, None] * K + bins_d.long()).reshape(-1)
    want = torch.zeros((F * K, 2), dtype=torch.int64, device=v.device)
    for k in range(2):
        want[:, k].index_add_(0, idx, m[k * M:(k + 1) * M].repeat(F))
    return want, torch.bincount(idx, minlength=F * K)


def sm_count_of(dev) -> int:
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The slowest rank's value (the timing rule for N > 1); identity on one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, steps: int, world: int, seconds_max: float) -> float:
    """Aggregate throughput over all ranks: units every rank processed / the slowest rank's time."""
    return units_per_rank * steps * world / seconds_max


def make_inputs(cfg: dict):
    p, q = synth.gen_primes(cfg["n_bits"], cfg["seed"])
    n = p * q
    gh = synth.gen_gh(cfg["M"], cfg.get("data_seed", cfg["seed"]))
    r = synth.gen_r(n, cfg["n_bits"], 2 * cfg["M"], cfg["seed"], p, q)
    bins = synth.make_bins(cfg)
    return p, q, gh, r, bins


# ----------------------------------------------------------------------------
# CPU oracle arm (reference and cpu_baseline)

def _oracle_sample_work(args):
    """The oracle's share of one step for a few samples: their encryptions,
    their histogram products, and a proportional number of decryptions."""
    import oracle
    n, p, q, ms, rs, ndec, F = args
    pub, priv = oracle.keypair(p, q)
    cts = [oracle.encrypt(pub, m, r) for m, r in zip(ms, rs)]
    acc = 1
    for _ in range(F):
        for c in cts:
            acc = oracle.add(pub, acc, c)
    for j in range(ndec):
        oracle.decrypt(priv, cts[j % len(cts)])
    return len(cts)


def oracle_rate(cfg, p, q, gh, r, samples: int, steps: int = 1):
    """Runs the oracle over `samples` samples per step on all host cores;
    returns (enc/s, wall seconds, cores)."""
    import multiprocessing as mp
    import oracle
    cores = len(os.sched_getaffinity(0))
    n = p * q
    M, F, K = cfg["M"], cfg["F"], cfg["K"]
    cells = F * K * 2
    ms = [oracle.encode(x) for x in np.concatenate([gh[0][:samples], gh[1][:samples]])]
    rs = synth.limbs_to_ints(np.concatenate([r[:samples], r[M:M + samples]]))
    ndec = max(1, round(cells * samples / M))
    nw = min(cores, 2 * samples)
    chunks = [list(range(i, 2 * samples, nw)) for i in range(nw)]
    per = [(n, p, q, [ms[i] for i in c], [rs[i] for i in c], (ndec if k == 0 else 0), F)
           for k, c in enumerate(chunks) if c]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(per)) as pool:
        pool.map(_oracle_sample_work, [(n, p, q, [ms[0]], [rs[0]], 0, 1)] * len(per))  # warm the workers
        t0 = time.perf_counter()
        done = 0
        for _ in range(steps):
            done += sum(pool.map(_oracle_sample_work, per))
        wall = time.perf_counter() - t0
    return done / wall, wall, len(per), ndec


def _oracle_op_worker(args):
    """Times one oracle operation type on a few inputs; returns (ops, seconds)."""
    import oracle
    op, p, q, vals = args
    pub, priv = oracle.keypair(p, q)
    t0 = time.perf_counter()
    if op == "encrypt":
        for m, r in vals:
            oracle.encrypt(pub, m, r)
    elif op == "mult":
        acc = 1
        for c in vals:
            acc = oracle.add(pub, acc, c)
    elif op == "decrypt":
        for c in vals:
            oracle.decrypt(priv, c)
    elif op == "decrypt_crt":
        for c in vals:
            oracle.decrypt_crt(priv, c)
    return len(vals), time.perf_counter() - t0


def run_oracle_rates(args):
    """Oracle rates per operation and key size, one core and all host cores, on
    bounded seeded samples, with the per-workload extrapolation (context only)."""
    import multiprocessing as mp
    import random as pyrandom
    cores = len(os.sched_getaffinity(0))
    per_core = {1024: 6, 2048: 3, 3072: 2}
    out = {"cores": cores, "rates": {}}
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        for nb in (1024, 2048, 3072):
            p, q = synth.gen_primes(nb, 7)
            n = p * q
            rng = pyrandom.Random(nb)
            import oracle
            pub = oracle.PublicKey(n)
            k = per_core[nb]
            enc_in = [(rng.randrange(1 << 25), rng.randrange(1, n)) for _ in range(k)]
            cts = [oracle.encrypt(pub, m, r) for m, r in enc_in]
            mult_in = [rng.randrange(1, n * n) for _ in range(2000)]
            rates = {}
            for op, vals in (("encrypt", enc_in), ("mult", mult_in), ("decrypt", cts), ("decrypt_crt", cts)):
                n1, t1 = _oracle_op_worker((op, p, q, vals))
                res = pool.map(_oracle_op_worker, [(op, p, q, vals)] * cores)
                wall = max(t for _, t in res)
                rates[op] = {"one_core_per_s": n1 / t1, "all_cores_per_s": sum(c for c, _ in res) / wall}
            out["rates"][nb] = rates
    r2 = out["rates"][2048]
    lv = synth.CONFIGS["level"]
    out["extrapolated_level_step_s_all_cores"] = (2 * lv["M"] / r2["encrypt"]["all_cores_per_s"] +
                                                  2 * lv["M"] * lv["F"] / r2["mult"]["all_cores_per_s"] +
                                                  lv["F"] * lv["K"] * 2 / r2["decrypt"]["all_cores_per_s"])
    out["note"] = "oracle as it stands (lambda-form decrypt is the definition); bounded samples; context only"
    emit_json(out)


def run_reference(args, cfg):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    p, q, gh, r, bins = make_inputs(cfg)
    samples = 16
    _ = oracle_rate(cfg, p, q, gh, r, 2, 1)  # warm-up run
    rate, wall, cores, ndec = oracle_rate(cfg, p, q, gh, r, samples, args.steps)
    sample = (f"per step {samples} samples of the '{args.config}' workload: {2 * samples} encryptions, "
              f"{2 * samples * cfg['F']} histogram products, {ndec} decryptions (lambda form)")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "enc/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "python-int",
        "data": "synthetic", "config": workload_config(args.config, cfg),
        "cpu_baseline": {"value": rate, "unit": "enc/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": "enc/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit_json(line)


# ----------------------------------------------------------------------------
# secure horizontal pattern (CKKS)

METRIC_H = "CKKS secure-horizontal rounds/s (clients encrypt local G/H histograms, server adds, client decrypts)"


def horizontal_inputs(cfg, nodes: int = 1):
    """Local histograms packed into complex slots (G real, H imaginary), the key
    material and every client's encryption randomness (all seeded).  Plaintext
    order [client][node][message]; `nodes` > 1 repeats the node's histograms
    (the histograms of one tree level) with fresh randomness per plaintext."""
    log_n, clients, F, K = cfg["log_n"], cfg["clients"], cfg["F"], cfg["K"]
    N = 1 << log_n
    slots = N // 2
    cells = F * K
    msgs = -(-cells // slots)
    hist = synth.horizontal_histograms(cfg["M"], F, K, clients, cfg["seed"])
    flat = np.zeros((clients, 1, msgs * slots, 2))
    flat[:, 0, :cells] = hist.reshape(clients, cells, 2)
    flat = np.repeat(flat, nodes, axis=1).reshape(clients * nodes * msgs, slots, 2)
    q = synth.ckks_prime(log_n)
    seed = cfg["seed"]
    key = (synth.ckks_secret(N, seed), synth.ckks_uniform(N, q, seed), synth.ckks_gaussian(N, seed, 1))
    B = clients * nodes * msgs
    rnd = (synth.ckks_ternary((B, N), seed, 2), synth.ckks_gaussian((B, N), seed, 3),
           synth.ckks_gaussian((B, N), seed, 4))
    return N, q, msgs, cells, hist, flat, key, rnd


def horizontal_config(cfg, msgs):
    return {"workload": f"secure horizontal round: {cfg['clients']} clients, {cfg['M']:,} samples split evenly, "
                        f"J x K = {cfg['F']} x {cfg['K']} G/H histograms packed into {msgs} plaintexts per client "
                        f"(N = {1 << cfg['log_n']}, one 60-bit prime, scale 2^{cfg['scale_bits']}); step = "
                        "encode + encrypt every client's plaintexts, server sum, decrypt + decode",
            "clients": cfg["clients"], "M": cfg["M"], "F": cfg["F"], "K": cfg["K"], "N": 1 << cfg["log_n"],
            "l2": "L2 flushed (256 MB write) before every timed step; steps timed one by one, each after "
                  "a short device-side delay that keeps the host's launch latency out of the interval",
            "parallelism": "replica per GPU"}


def _horizontal_oracle_sample(cfg):
    """The oracle on one client plaintext (encode + encrypt) and one aggregate
    (sum of the clients' ciphertexts, decrypt + decode); returns seconds per
    round scaled to the whole round and the seconds spent."""
    from oracle import ckks as ock
    N, q, msgs, cells, hist, flat, (s, a, e), (v, e0, e1) = horizontal_inputs(cfg)
    scale = 2.0 ** cfg["scale_bits"]
    clients = cfg["clients"]
    b = ock.keygen(s, a, e, q)
    t0 = time.perf_counter()
    m = ock.encode(flat[0, :, 0] + 1j * flat[0, :, 1], N, scale)
    c = ock.encrypt(b, a, m, v[0], e0[0], e1[0], q)
    t1 = time.perf_counter()
    tot = c
    for _ in range(clients - 1):
        tot = ock.add(tot, c, q)
    t2 = time.perf_counter()
    ock.decode(ock.centre(ock.decrypt(tot, s, q), q), N, scale)
    t3 = time.perf_counter()
    per_round = clients * msgs * (t1 - t0) + msgs * (t2 - t1) + msgs * (t3 - t2)
    return per_round, t3 - t0


# algorithmic work of the CKKS kernels, per plaintext (N = 2n coefficients)
def ckks_fft_flop(N: int) -> int:
    """encode/decode: a length-n complex radix-2 FFT (5 n log2 n FLOP) plus the
    twist by omega^k (6 n) and the scaling (2 n)."""
    n = N // 2
    return 5 * n * (n.bit_length() - 1) + 8 * n


def ckks_encrypt_imad(N: int) -> int:
    """k_encrypt: forward NTT of v (N/2 log2 N Montgomery products), 4 N in the
    pointwise products, two inverse NTTs (+ N for the N^-1 fold); 20 IMAD
    halves per 64-bit Montgomery product (a b: 4 limb products, m = lo q': 2,
    m q: 4; 2 halves each)."""
    lg = N.bit_length() - 1
    mm = (N // 2) * lg + 4 * N + 2 * (N // 2) * lg + N
    return 20 * mm


def ckks_decrypt_imad(N: int) -> int:
    """k_decrypt: forward NTT of c1, 2 N in the pointwise product, one inverse
    NTT (+ N/2 for the N^-1 fold); 20 IMAD halves per Montgomery product."""
    lg = N.bit_length() - 1
    return 20 * ((N // 2) * lg + 2 * N + (N // 2) * lg + N // 2)


class _HorizontalCase:
    """Device buffers and one captured CUDA graph of a horizontal round over
    `nodes` node histograms."""

    def __init__(self, cfg, ctx, nodes, dev, torch):
        clients = cfg["clients"]
        N, q, msgs, cells, hist, flat, (s, a, e), (v, e0, e1) = horizontal_inputs(cfg, nodes)
        self.N, self.msgs, self.cells, self.hist, self.nodes = N, msgs, cells, hist, nodes
        B = clients * nodes * msgs
        self.B = B
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        self.h_in = [pin(flat[..., 0]), pin(flat[..., 1]), pin(v), pin(e0), pin(e1)]
        self.d_in = [t.to(dev) for t in self.h_in]
        self.s_d = torch.from_numpy(s).to(dev)
        self.a_d = torch.from_numpy(a.view(np.int64)).to(dev)
        self.b_d = ctx.keygen(self.s_d, self.a_d, torch.from_numpy(e).to(dev))
        # the clients' keys are fixed across rounds: transforms taken once, outside the round
        ctx.prepare_public_key(self.b_d, self.a_d)
        ctx.prepare_secret_key(self.s_d)
        self.m = torch.empty(B, N, dtype=torch.int64, device=dev)
        self.c = torch.empty(B, 2, N, dtype=torch.int64, device=dev)
        self.tot = torch.empty(nodes * msgs, 2, N, dtype=torch.int64, device=dev)
        self.h_out = torch.empty(2, nodes * msgs, N // 2, dtype=torch.float64).pin_memory()
        self.ctx, self.clients, self.torch = ctx, clients, torch
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        self.out = {}
        torch.cuda.synchronize()  # inputs and the key are ready before any other stream uses them

    def step(self, mark=False, copies=False):
        ctx, ev, k = self.ctx, self.ev, self.nodes * self.msgs
        if copies:
            for dst, src in zip(self.d_in, self.h_in):
                dst.copy_(src, non_blocking=True)
        re, im, v, e0, e1 = self.d_in
        if mark:
            ev[0].record()
        self.m = ctx.encode(re, im)
        if mark:
            ev[1].record()
        ctx.encrypt_prepared(self.m, v, e0, e1, out=self.c)
        if mark:
            ev[2].record()
        ctx.sum([self.c[i * k:(i + 1) * k] for i in range(self.clients)], out=self.tot)
        if mark:
            ev[3].record()
        self.d = ctx.decrypt_prepared(self.tot)
        if mark:
            ev[4].record()
        self.out["re"], self.out["im"] = ctx.decode(self.d)
        if mark:
            ev[5].record()
        if copies:
            self.h_out[0].copy_(self.out["re"], non_blocking=True)
            self.h_out[1].copy_(self.out["im"], non_blocking=True)

    def phase(self, i):
        """Phase i of the round alone (0 encode, 1 encrypt, 2 sum, 3 decrypt,
        4 decode) on the buffers of an earlier step."""
        ctx, k = self.ctx, self.nodes * self.msgs
        re, im, v, e0, e1 = self.d_in
        if i == 0:
            self.m = ctx.encode(re, im)
        elif i == 1:
            ctx.encrypt_prepared(self.m, v, e0, e1, out=self.c)
        elif i == 2:
            ctx.sum([self.c[j * k:(j + 1) * k] for j in range(self.clients)], out=self.tot)
        elif i == 3:
            self.d = ctx.decrypt_prepared(self.tot)
        else:
            self.out["re"], self.out["im"] = ctx.decode(self.d)

    def capture(self, copies=False):
        """Captures one round (warm: scratch already sized) into a CUDA graph;
        returns (graph, library kernels in it)."""
        from paper_2504_03909_b300 import native
        torch = self.torch
        g = torch.cuda.CUDAGraph()
        n0 = native.lib().paillier_launch_count()
        with torch.cuda.graph(g):
            self.step(copies=copies)
        return g, int(native.lib().paillier_launch_count() - n0)

    def check(self, scale):
        got = np.stack([self.out["re"].cpu().numpy(), self.out["im"].cpu().numpy()], -1)
        got = got.reshape(self.nodes, -1, 2)[:, :self.cells]
        want = self.hist.sum(0).reshape(-1, 2)
        err = float(np.abs(got - want[None]).max())
        bound = self.clients * self.N * (0.5 + 19 * (2 * self.N + 1)) / scale
        if not err <= bound + 1e-9 * np.abs(want).max():
            raise RuntimeError(f"horizontal round error {err} above the bound {bound}")
        return err, bound


def run_horizontal(args, cfg):
    import torch
    from paper_2504_03909_b300 import ckks as G, native

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    clients = cfg["clients"]
    scale = 2.0 ** cfg["scale_bits"]
    q = synth.ckks_prime(cfg["log_n"])
    ctx = G.Context(cfg["log_n"], q, scale)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # measured peaks (same process, same clocks)
    peaks = {}
    for name, fn, extra in (("fp64_flop_s", "paillier_fp64_peak", ()), ("imad_s", "paillier_imad_peak", (1,))):
        rate, el = native.C.c_double(0), native.C.c_double(0)
        native.call(fn, *extra, 1000.0, native.C.byref(rate), native.C.byref(el), torch.cuda.current_stream().cuda_stream)
        peaks[name] = rate.value

    def measure(nodes, steps):
        """Warm-up, correctness check, captured graph; timed replays (one by one,
        L2 flushed before each) and per-phase times from an eager pass."""
        case = _HorizontalCase(cfg, ctx, nodes, dev, torch)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                case.step()
            stream.synchronize()
            err, bound = case.check(scale)
            g, launches = case.capture()
            ge, _ = case.capture(copies=True)
            t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            phases = np.zeros(5)
            for _ in range(steps):  # per-phase device times: each phase alone, as the round is timed
                for i in range(5):
                    flush.fill_(1)
                    torch.cuda._sleep(400_000)
                    t0e.record()
                    case.phase(i)
                    t1e.record()
                    stream.synchronize()
                    phases[i] += t0e.elapsed_time(t1e)
            barrier()
            total = 0.0
            with ClockSampler(local) as clk:
                # keep the GPU busy long enough for the sampler's first readings
                t_end = time.perf_counter() + 0.6
                while time.perf_counter() < t_end:
                    for _ in range(50):
                        g.replay()
                    stream.synchronize()
                for _ in range(steps):
                    flush.fill_(1)
                    # a bounded device-side delay (about 0.2 ms of spinning): the host enqueues the
                    # start event and the round meanwhile, so its launch latency stays out of the
                    # device-timed interval (the e2e number below keeps it)
                    torch.cuda._sleep(400_000)
                    t0e.record()
                    g.replay()
                    t1e.record()
                    stream.synchronize()
                    total += t0e.elapsed_time(t1e) / 1e3
            e2e = 0.0
            for _ in range(steps):
                flush.fill_(1)
                t0e.record()
                ge.replay()
                t1e.record()
                stream.synchronize()
                e2e += t0e.elapsed_time(t1e) / 1e3
            case.check(scale)
        return case, total, e2e, phases / steps, launches, err, bound, clk.summary()

    case, total, e2e, ph, launches, err, bound, clk = measure(args.nodes, args.steps)
    total = max_over_ranks(total, dist, dev)
    e2e = max_over_ranks(e2e, dist, dev)
    lvl = None
    if args.nodes == 1:
        lvl_case, lt, le, lph, _, _, _, _ = measure(32, args.steps)
        lvl = (lvl_case, lt, lph)

    N, B, msgs = case.N, case.B, case.msgs
    names = ["encode", "encrypt", "sum", "decrypt", "decode"]
    fft_flop = ckks_fft_flop(N)
    enc_imad = ckks_encrypt_imad(N)

    def ctas(polys):
        """CTAs of a launch over `polys` polynomials: a cluster of 8 per polynomial
        up to 64 polynomials (N >= 1024), else one each."""
        return polys * 8 if cfg["log_n"] >= 10 and polys <= 64 else polys

    def roof(phases, b):
        """Dominant phase and its achieved rate against the measured peak."""
        i = int(np.argmax(phases))
        if names[i] in ("encode", "decode"):
            work, peak, meas, unit, kern = fft_flop * (b if names[i] == "encode" else b // clients), \
                FP64_NOMINAL_TFLOPS * 1e12, peaks["fp64_flop_s"], "TFLOP/s", f"k_{names[i]} (float64 FFT)"
            src = "B300 nominal float64 rate (1.25 TFLOP/s)"
        elif names[i] in ("encrypt", "decrypt"):
            per = enc_imad if names[i] == "encrypt" else ckks_decrypt_imad(N)
            work, peak, meas, unit, kern = per * (b if names[i] == "encrypt" else b // clients), \
                imad_peak_derived(sm_count_of(dev)), peaks["imad_s"], "TIMAD/s", f"k_{names[i]} (64-bit Montgomery NTT)"
            src = "derived: SMs x 64 IMAD lanes/clk/SM x 2032 MHz max SM clock"
        else:
            return None
        ach = work / (phases[i] * 1e-3)
        return {"bound": "alu", "kernel": kern, "achieved": ach / 1e12, "peak": peak / 1e12, "unit": unit,
                "frac": ach / peak, "traffic": None, "work_per_launch": work, "launch_ms": phases[i],
                "ctas": ctas(b if names[i] in ("encode", "encrypt") else b // clients), "sms": sm_count_of(dev),
                "peak_source": src, "peak_measured": meas / 1e12, "frac_of_measured": ach / meas,
                "measured_note": "project microbenchmark in the same run (paillier_fp64_peak / paillier_imad_peak "
                                 "mad.wide)"}

    line = {
        "metric": METRIC_H, "value": whole_job_rate(args.nodes, args.steps, world, total),
        "unit": "rounds/s" if args.nodes == 1 else "node-rounds/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64",
        "data": "synthetic (seeded local histograms of logistic g/h over N(0,1) features, quantile-binned)",
        "config": dict(horizontal_config(cfg, msgs), nodes=args.nodes, graph="one CUDA graph per round"),
        "phases_ms_per_step": dict(zip(names, ph.tolist())),
        "phases_note": "each phase alone on the device after the L2 flush and a short device-side delay "
                       "(its inputs cold, as at the start of a round)",
        "max_abs_error": err, "error_bound": bound,
        "roofline": roof(ph, B),
        "clocks": clk,
        "e2e": {"value": whole_job_rate(args.nodes, args.steps, world, e2e), "unit": "rounds/s",
                "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in case.h_in),
                "d2h_bytes_per_step": case.h_out.numel() * 8},
        "gpu_launches": launches * args.steps,
        "peaks_measured": {"fp64_TFLOP_s": peaks["fp64_flop_s"] / 1e12, "imad_T_s": peaks["imad_s"] / 1e12},
    }
    if lvl is not None:
        lc, lt, lph = lvl
        line["level_32_nodes"] = {"rounds_per_s": 32 * args.steps / lt, "ms_per_level": 1e3 * lt / args.steps,
                                  "phases_ms": dict(zip(names, lph.tolist())), "roofline": roof(lph, lc.B),
                                  "note": "32 node histograms (a depth-6 tree's last level) in one batch"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_round, wall = _horizontal_oracle_sample(cfg)
        line["cpu_baseline"] = {"value": 1.0 / per_round, "unit": "rounds/s", "cores": 1, "kind": "oracle",
                                "sample": f"one client plaintext (encode + encrypt) and one aggregate (sum of "
                                          f"{clients}, decrypt + decode), scaled to the round's {clients * msgs} "
                                          f"and {msgs}; {wall:.1f} s wall"}
    if dist is not None:
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_reference_horizontal(args, cfg):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    N, q, msgs, *_ = horizontal_inputs(cfg)
    t = [_horizontal_oracle_sample(cfg) for _ in range(args.steps)]
    per_round = sum(x[0] for x in t) / len(t)
    rate = 1.0 / per_round
    sample = (f"per step one client plaintext (encode + encrypt) and one aggregate (sum, decrypt + decode) of the "
              f"horizontal round, scaled to its {cfg['clients'] * msgs} plaintexts and {msgs} aggregates")
    line = {
        "impl": "reference", "metric": METRIC_H, "value": rate, "unit": "rounds/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_round, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "python-int+f64", "data": "synthetic",
        "config": horizontal_config(cfg, msgs),
        "cpu_baseline": {"value": rate, "unit": "rounds/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": "rounds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit_json(line)


def run_sharded(args, cfg):
    """N > 1: one level job split over the ranks (paper_2504_03909_b300.shard):
    rank k encrypts samples [k M / N, (k + 1) M / N), an NCCL all-gather hands
    every ciphertext to every rank, rank k aggregates and decrypts the features
    [k F / N, (k + 1) F / N), and the decrypted sums are gathered.  The total
    work is that of one level whatever N (strong scaling)."""
    import torch
    import torch.distributed as dist
    from paper_2504_03909_b300 import native, paillier as P, shard

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if "MASTER_ADDR" not in os.environ:  # one rank started without torchrun (--shard)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(29500 + os.getpid() % 1000), RANK="0",
                          WORLD_SIZE="1")
    dev = torch.device("cuda", local)
    dist.init_process_group("nccl", device_id=dev)
    M, F, K, n_bits = cfg["M"], cfg["F"], cfg["K"], cfg["n_bits"]
    L = n_bits // 32
    p, q, gh, r, bins = make_inputs(cfg)
    key = P.Key.from_primes(n_bits, p, q)
    s_lo, s_hi = shard.block_range(M, world, rank)
    f_lo, f_hi = shard.block_range(F, world, rank)
    ms_, fk = s_hi - s_lo, f_hi - f_lo
    # this rank's inputs: its samples' g/h and randomness, its features' bins (all samples)
    h_v = torch.from_numpy(np.concatenate([gh[0, s_lo:s_hi], gh[1, s_lo:s_hi]])).pin_memory()
    r32 = r.view(np.int32).reshape(2 * M, L)
    h_r = torch.from_numpy(np.concatenate([r32[s_lo:s_hi], r32[M + s_lo:M + s_hi]])).pin_memory()
    h_bins = torch.from_numpy(np.ascontiguousarray(bins[f_lo:f_hi])).pin_memory()
    h_node = torch.zeros(M, dtype=torch.int32).pin_memory()
    v, r_d, bins_d, node = h_v.to(dev), h_r.to(dev), h_bins.to(dev), h_node.to(dev)
    ct_loc = torch.empty((2 * ms_, 2 * L), dtype=torch.int32, device=dev)
    hist = torch.empty((1, fk, K, 2, 2 * L), dtype=torch.int32, device=dev)
    cnt = torch.empty((1, fk, K), dtype=torch.int32, device=dev)
    sums = torch.empty((1, fk, K, 2), dtype=torch.int64, device=dev)
    cnt2 = torch.empty((1, fk, K, 2), dtype=torch.int32, device=dev)
    out = torch.empty((1, fk, K, 2), dtype=torch.float64, device=dev)
    h_out = torch.empty(out.shape, dtype=torch.float64).pin_memory()

    def encrypt(_range):
        P.encrypt(key, P.encode(v), r_d, out=ct_loc)
        return ct_loc.view(2, ms_, 2 * L)

    def prepare(ct):
        return P.ct_prepare(key, ct.reshape(2 * M, 2 * L)).view(2, M, 2 * L)

    def aggregate(ctm, a, b):
        return P.hist_aggregate(key, ctm, bins_d, node, 1, K, hist=hist, count=cnt)

    def decrypt(h):
        P.decrypt_u64(key, h.view(-1, 2 * L), out=sums.view(-1))
        cnt2.copy_(cnt.unsqueeze(-1).expand(1, fk, K, 2))
        P.decode(sums, cnt2, out=out)
        return sums

    ops = shard.LevelOps(encrypt=encrypt, prepare=prepare, aggregate=aggregate, decrypt=decrypt,
                         empty_rows=lambda n: torch.empty((2, n, 2 * L), dtype=torch.int32, device=dev))

    def step():
        return shard.run_level(ops, dist, world, rank, M, F)

    def barrier():
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    P.sync()
    native.call("paillier_profile", 1)
    n0 = native.lib().paillier_launch_count()
    barrier()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            full = step()[0]
        e1.record()
        barrier()
    launches = native.lib().paillier_launch_count() - n0
    prof = {}
    for kname in ("modexp_enc1", "modexp_enc"):
        tot_ms, cnt_l = native.C.c_double(0), native.C.c_longlong(0)
        native.call("paillier_profile_read", kname.encode(), native.C.byref(tot_ms), native.C.byref(cnt_l))
        prof[kname] = (tot_ms.value, cnt_l.value)
    native.call("paillier_profile", 0)
    elapsed = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
    # roofline of the dominant launch (the second encryption stage) on this rank's share, slowest rank
    lanes_enc, w = P.get_config(key, native.OP_ENCRYPT)
    imad1, imad2 = enc_imad_stages(n_bits, w, p, q, lanes_enc)
    split = prof["modexp_enc1"][1] > 0
    launch_ms = max_over_ranks(prof["modexp_enc"][0] / max(1, prof["modexp_enc"][1]), dist, dev)
    imad_launch = 2 * ms_ * (imad2 if split else imad1 + imad2)
    peak = imad_peak_derived(sm_count_of(dev))
    P.sync()
    # untimed: the gathered sums equal the plaintext sums of every feature
    v_all = torch.from_numpy(gh.reshape(-1).copy()).to(dev)
    want, _ = plaintext_root_sums(P, torch, v_all, torch.from_numpy(bins).to(dev), M, F, K)
    if not torch.equal(full.view(F * K, 2), want):
        raise RuntimeError("sharded sums differ from the plaintext sums")
    # end to end: each rank's input slices in from pinned host memory, its decoded block out
    h2d_rank = h_v.numel() * 4 + h_r.numel() * 4 + h_bins.numel() + h_node.numel() * 4
    d2h_rank = h_out.numel() * 8
    tot = torch.tensor([h2d_rank, d2h_rank], dtype=torch.float64, device=dev)
    dist.all_reduce(tot)
    barrier()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record()
    for _ in range(args.steps):
        v.copy_(h_v, non_blocking=True)
        r_d.copy_(h_r, non_blocking=True)
        bins_d.copy_(h_bins, non_blocking=True)
        node.copy_(h_node, non_blocking=True)
        step()
        h_out.copy_(out, non_blocking=True)
    e3.record()
    barrier()
    e2e_s = max_over_ranks(e2.elapsed_time(e3) / 1e3, dist, dev)
    launches_max = max_over_ranks(float(launches), dist, dev)
    line = {
        "metric": METRIC, "value": 2 * M * args.steps / elapsed, "unit": "enc/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded: logistic g/h, Bernoulli(0.3) labels, N(0,1) features quantile-binned)",
        "config": dict(workload_config(args.config, cfg),
                       parallelism=f"sharded over {world} GPUs: samples for encryption, NCCL all-gather of the "
                                   "ciphertext rows, features for aggregation and decryption, gather of the sums"),
        "clocks": clk.summary(),
        "e2e": {"value": 2 * M * args.steps / e2e_s, "unit": "enc/s", "h2d_bytes_per_step": int(tot[0].item()),
                "d2h_bytes_per_step": int(tot[1].item())},
        "gpu_launches": int(launches_max * world),
        "roofline": {"bound": "alu",
                     "kernel": "k_modexp (encryption, second stage: z^x mod x^2)" if split else "k_modexp (encryption)",
                     "achieved": imad_launch / (launch_ms * 1e-3) / 1e12, "peak": peak / 1e12, "unit": "TIMAD/s",
                     "frac": imad_launch / (launch_ms * 1e-3) / peak,
                     "traffic": 2 * ms_ * TRAFFIC_PER_ENC[(n_bits, w)] if (n_bits, w) in TRAFFIC_PER_ENC else None,
                     "peak_source": "derived: SMs x 64 IMAD lanes/clk/SM (4 sub-partitions x 16) x 2032 MHz max SM "
                                    "clock", "launch_ms": launch_ms, "imad_per_launch": imad_launch,
                     "note": "per rank (its share of the encryptions), slowest rank's launch"},
        "verified": f"gathered sums == plaintext sums of the encoded values, all {F * K * 2} cells (untimed)",
    }
    dist.destroy_process_group()
    if rank == 0:
        emit_json(line)


def workload_config(name, cfg):
    desc = {
        "level": "one tree level: 250,000 samples x 30 features (N(0,1), quantile-binned) x 256 bins, 2048-bit n, "
                 "root node; encrypt 500k g/h, histogram 30x256x2, CRT-decrypt 15,360 cells",
        "toy": "toy: 1,000 samples x 8 features x 16 bins, 1024-bit n, root node",
        "level_small": "small case of the level kernels: 8,192 samples x 30 features x 256 bins, 2048-bit n, root",
    }.get(name, name)
    return {"workload": desc, "M": cfg["M"], "F": cfg["F"], "K": cfg["K"], "n_bits": cfg["n_bits"],
            "nodes": 1, "l2": "inputs larger than L2 (r 128 MB, ciphertexts 256 MB at 2048-bit)",
            "parallelism": "replica per GPU"}


# ----------------------------------------------------------------------------

def run_ours(args, cfg):
    import torch
    from paper_2504_03909_b300 import native, paillier as P

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    M, F, K, n_bits = cfg["M"], cfg["F"], cfg["K"], cfg["n_bits"]
    L = n_bits // 32
    p, q, gh, r, bins = make_inputs(cfg)
    key = P.Key.from_primes(n_bits, p, q)

    # host (pinned) and device copies of the inputs
    h_v = torch.from_numpy(gh.reshape(-1).copy()).pin_memory()
    h_r = torch.from_numpy(r.view(np.int32)).pin_memory()
    h_bins = torch.from_numpy(bins).pin_memory()
    h_node = torch.zeros(M, dtype=torch.int32).pin_memory()
    v = h_v.to(dev)
    r_d = h_r.to(dev)
    bins_d = h_bins.to(dev)
    node = h_node.to(dev)
    ct = torch.empty((2 * M, 2 * L), dtype=torch.int32, device=dev)
    ctm = torch.empty_like(ct)
    hist = torch.empty((1, F, K, 2, 2 * L), dtype=torch.int32, device=dev)
    cnt = torch.empty((1, F, K), dtype=torch.int32, device=dev)
    sums = torch.empty((1, F, K, 2), dtype=torch.int64, device=dev)
    cnt2 = torch.empty((1, F, K, 2), dtype=torch.int32, device=dev)
    out = torch.empty((1, F, K, 2), dtype=torch.float64, device=dev)
    h_out = torch.empty(out.shape, dtype=torch.float64).pin_memory()

    def step():
        m = P.encode(v)
        P.encrypt(key, m, r_d, out=ct)
        P.ct_prepare(key, ct, out=ctm)
        P.hist_aggregate(key, ctm.view(2, M, 2 * L), bins_d, node, 1, K, hist=hist, count=cnt)
        P.decrypt_u64(key, hist.view(-1, 2 * L), out=sums.view(-1))
        cnt2.copy_(cnt.unsqueeze(-1).expand(1, F, K, 2))
        P.decode(sums, cnt2, out=out)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # measured integer multiply-add peaks (same process, same clocks)
    peaks = {}
    for mix, name in ((0, "carry_rows"), (1, "mad_wide"), (2, "lo_hi")):
        rate = native.C.c_double(0)
        el = native.C.c_double(0)
        native.call("paillier_imad_peak", mix, 1500.0, native.C.byref(rate), native.C.byref(el),
                    torch.cuda.current_stream().cuda_stream)
        peaks[name] = rate.value

    for _ in range(args.warmup):
        step()
    P.sync()

    native.call("paillier_profile", 1)
    n0 = native.lib().paillier_launch_count()
    barrier()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        barrier()
    launches = native.lib().paillier_launch_count() - n0
    elapsed = e0.elapsed_time(e1) / 1e3
    prof = {}
    for kname in ("encode", "modexp_enc1", "modexp_enc", "enc_crt", "to_mont", "hist_count", "hist_scan", "feat_scan",
                  "hist_scatter", "seg_product", "combine", "modexp_dec", "dec_crt", "decode"):
        tot = native.C.c_double(0)
        cntl = native.C.c_longlong(0)
        native.call("paillier_profile_read", kname.encode(), native.C.byref(tot), native.C.byref(cntl))
        prof[kname] = (tot.value, cntl.value)
    native.call("paillier_profile", 0)
    P.sync()
    elapsed = max_over_ranks(elapsed, dist, dev)

    # end to end through the public API with pinned host buffers
    h2d = h_v.numel() * 4 + h_r.numel() * 4 + h_bins.numel() + h_node.numel() * 4
    d2h = h_out.numel() * 8
    e2e_steps = max(1, args.steps)
    barrier()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record()
    for _ in range(e2e_steps):
        v.copy_(h_v, non_blocking=True)
        r_d.copy_(h_r, non_blocking=True)
        bins_d.copy_(h_bins, non_blocking=True)
        node.copy_(h_node, non_blocking=True)
        step()
        h_out.copy_(out, non_blocking=True)
    e3.record()
    barrier()
    e2e_s = e2.elapsed_time(e3) / 1e3
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    P.sync()
    want, want_cnt = plaintext_root_sums(P, torch, v, bins_d, M, F, K)
    if not (torch.equal(sums.view(F * K, 2), want) and torch.equal(cnt.view(-1).long(), want_cnt)):
        raise RuntimeError("decrypted root histogram differs from the plaintext sums")

    # the same step with g/h packing (one plaintext enc(g) + 2^B enc(h) per
    # sample, a decrypt-count reduction the paper does not use): reported
    # beside the headline, which keeps the paper's two ciphertexts per sample
    gh_line = None
    if args.gh_bits:
        B = args.gh_bits
        g_d, h_d = v[:M], v[M:]
        m2 = torch.empty((M, 2), dtype=torch.int64, device=dev)
        ct1 = torch.empty((M, 2 * L), dtype=torch.int32, device=dev)
        ctm1 = torch.empty_like(ct1)
        hist1 = torch.empty((1, F, K, 2 * L), dtype=torch.int32, device=dev)
        sums1 = torch.empty((F * K, 2), dtype=torch.int64, device=dev)

        def step_gh():
            P.encode_gh(g_d, h_d, B, out=m2)
            P.encrypt_gh(key, m2, r_d[:M], out=ct1)
            P.ct_prepare(key, ct1, out=ctm1)
            P.hist_aggregate_gh(key, ctm1, bins_d, node, 1, K, hist=hist1, count=cnt)
            P.decrypt_gh(key, hist1.view(-1, 2 * L), B, out=sums1)
            cnt2.copy_(cnt.unsqueeze(-1).expand(1, F, K, 2))
            P.decode(sums1.view(1, F, K, 2), cnt2, out=out)

        for _ in range(args.warmup):
            step_gh()
        P.sync()
        if not torch.equal(sums1.view(-1), sums.view(-1)):
            raise RuntimeError("g/h-packed sums differ from the two-ciphertext sums")
        barrier()
        e4 = torch.cuda.Event(enable_timing=True)
        e5 = torch.cuda.Event(enable_timing=True)
        e4.record()
        for _ in range(args.steps):
            step_gh()
        e5.record()
        barrier()
        t_gh = max_over_ranks(e4.elapsed_time(e5) / 1e3, dist, dev)
        gh_line = {"gh_bits": B, "ms_per_step": 1e3 * t_gh / args.steps,
                   "values_per_s": whole_job_rate(2 * M, args.steps, world, t_gh),
                   "ciphertexts_per_s": whole_job_rate(M, args.steps, world, t_gh),
                   "note": "same step, one ciphertext per sample for g and h; sums checked equal"}

    units = 2 * M  # g and h values through the whole path per step and GPU
    value = whole_job_rate(units, args.steps, world, elapsed)
    def ms(k):
        return prof[k][0]

    phase = {
        "encode": ms("encode"),
        "encrypt": ms("modexp_enc1") + ms("modexp_enc") + ms("enc_crt"),
        "prepare": ms("to_mont"),
        "aggregate": sum(ms(k) for k in ("hist_count", "hist_scan", "feat_scan", "hist_scatter", "seg_product",
                                         "combine")),
        "decrypt": ms("modexp_dec") + ms("dec_crt"),
        "decode": ms("decode"),
    }
    phase = {k: v_ / args.steps for k, v_ in phase.items()}  # ms per step
    lanes_enc, w = P.get_config(key, native.OP_ENCRYPT)
    # encryption runs as one launch, or as two (first stage mod x, then the second mod x^2,
    # which dominates the step): the roofline is that of the dominant launch; the work is the
    # multiply-adds the kernels execute (squarings form each cross product once), the CIOS
    # count of the same schedules beside it
    imad1, imad2 = enc_imad_stages(n_bits, w, p, q, lanes_enc)
    cios1, cios2 = enc_imad_stages(n_bits, w, p, q, lanes_enc, cios=True)
    split = prof["modexp_enc1"][1] > 0
    enc_launch_ms = prof["modexp_enc"][0] / max(1, prof["modexp_enc"][1])
    imad_launch = units * (imad2 if split else imad1 + imad2)
    imad_launch_cios = units * (cios2 if split else cios1 + cios2)
    achieved = imad_launch / (enc_launch_ms * 1e-3)
    peak = imad_peak_derived(sm_count_of(dev))
    best_mix = max(peaks.values())
    first_stage = None
    if split:
        t1 = prof["modexp_enc1"][0] / max(1, prof["modexp_enc1"][1])
        first_stage = {"kernel": "k_modexp (encryption, first stage: (r mod x)^(x' mod (x - 1)) mod x)",
                       "achieved": units * imad1 / (t1 * 1e-3) / 1e12, "frac": units * imad1 / (t1 * 1e-3) / peak,
                       "launch_ms": t1, "imad_per_launch": units * imad1}
    # the encrypted histogram's segmented product: one product mod n^2 (2L limbs) per contribution
    t_seg = prof["seg_product"][0] / max(1, prof["seg_product"][1])
    agg_imad = M * F * 2 * mont_imad(2 * L)
    agg_rate = agg_imad / (t_seg * 1e-3)
    aggregate_roofline = {
        "bound": "alu", "kernel": "k_seg_product (one product mod n^2 per (sample, feature, g/h) contribution)",
        "achieved": agg_rate / 1e12, "peak": peak / 1e12, "unit": "TIMAD/s", "frac": agg_rate / peak,
        "frac_of_measured_best_mix": agg_rate / best_mix, "frac_of_carry_chain_mix": agg_rate / peaks["carry_rows"],
        "launch_ms": t_seg, "imad_per_launch": agg_imad,
        "dram_note": "ncu capture of the segmented product on 2 x 65,536 x 16 contributions: DRAM reads "
                     "about one pass over the ciphertexts, 3.6 GB/s, 0.05 % of peak: the pass is ALU-bound",
    }
    # the CRT decryption of the level's cells: c^(x - 1) mod x^2 per half, the
    # schedule's multiply-adds as executed and at the CIOS cost per product
    lanes_dec, w_dec = P.get_config(key, native.OP_DECRYPT)
    t_dec = prof["modexp_dec"][0] / max(1, prof["modexp_dec"][1])
    ndec = F * K * 2
    dec_exec = ndec * dec_imad(n_bits, w_dec, p, q, lanes_dec)
    dec_cios = ndec * dec_imad(n_bits, w_dec, p, q)
    decrypt_roofline = {
        "bound": "alu", "kernel": "k_modexp (decryption: c^(x - 1) mod x^2 per CRT half)",
        "achieved": dec_exec / (t_dec * 1e-3) / 1e12, "peak": peak / 1e12, "unit": "TIMAD/s",
        "frac": dec_exec / (t_dec * 1e-3) / peak, "frac_cios_count": dec_cios / (t_dec * 1e-3) / peak,
        "launch_ms": t_dec, "imad_per_launch": dec_exec, "imad_per_launch_cios_count": dec_cios,
        "cells": ndec, "lanes": lanes_dec, "window": w_dec,
    }
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "enc/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic (seeded: logistic g/h, Bernoulli(0.3) labels, N(0,1) features quantile-binned)",
        "config": workload_config(args.config, cfg),
        "phases_ms_per_step": phase,
        "enc_per_s": units / (phase["encrypt"] * 1e-3),
        "ct_mults_per_s": M * F * 2 / (phase["aggregate"] * 1e-3),
        "ct_mults_strict_per_step": 2 * F * (M - K),
        "decrypts_per_s": F * K * 2 / (phase["decrypt"] * 1e-3),
        "roofline": {
            "bound": "alu",
            "kernel": "k_modexp (encryption, second stage: z^x mod x^2)" if split else "k_modexp (encryption)",
            "achieved": achieved / 1e12,
            "peak": peak / 1e12,
            "unit": "TIMAD/s",
            "frac": achieved / peak,
            # DRAM bytes per encryption of this kernel version from an ncu capture of 16,384
            # encryptions (w = 6), scaled to this launch
            "traffic": units * TRAFFIC_PER_ENC.get((n_bits, w)) if (n_bits, w) in TRAFFIC_PER_ENC else None,
            "traffic_note": "ncu dram__bytes_read+write of a 16,384-encryption capture of this kernel "
                            "version, scaled by encryptions",
            "peak_source": "derived: SMs x 64 IMAD lanes/clk/SM (4 sub-partitions x 16) x 2032 MHz max SM clock",
            "sms": sm_count_of(dev),
            "peaks_measured_TIMAD_s": {k: v_ / 1e12 for k, v_ in peaks.items()},
            "frac_of_measured_best_mix": achieved / best_mix,
            "frac_of_carry_chain_mix": achieved / peaks["carry_rows"],
            "measured_note": "project microbenchmark paillier_imad_peak in the same run: carry_rows is the "
                             "instruction mix of the kernel's Montgomery rows",
            "imad_per_launch": imad_launch,
            "imad_per_launch_cios_count": imad_launch_cios,
            "frac_cios_count": imad_launch_cios / (enc_launch_ms * 1e-3) / peak,
            "imad_note": "imad_per_launch counts the multiply-add halves the kernel executes (separated-form "
                         "squarings form each cross product once); imad_per_launch_cios_count is the same schedule "
                         "at 4 L^2 + L per product",
            "launch_ms": enc_launch_ms,
            "first_stage": first_stage,
        },
        "aggregate_roofline": aggregate_roofline,
        "decrypt_roofline": decrypt_roofline,
        "clocks": clk.summary(),
        "e2e": {"value": whole_job_rate(units, e2e_steps, world, e2e_s), "unit": "enc/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "verified": f"decrypted root histogram == plaintext sums of the encoded values, all {F * K * 2} cells "
                    "and counts (untimed)",
    }
    if gh_line is not None:
        line["gh_packed"] = gh_line
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        samples = 48
        rate, wall, cores, ndec = oracle_rate(cfg, p, q, gh, r, samples, 1)
        line["cpu_baseline"] = {
            "value": rate, "unit": "enc/s", "cores": cores, "kind": "oracle",
            "sample": f"{samples} samples of the workload: {2 * samples} encryptions, {2 * samples * F} histogram "
                      f"products, {ndec} decryptions (lambda form); {wall:.1f} s wall"}
    if dist is not None:
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_batched(args, cfg, emit=True):
    """Depth-6 tree on the level data: encrypt once, then for every level the
    batched histogram (one captured graph, replayed per level) and the CRT
    decryption of all the level's cells; the per-node launch path is timed on
    the same levels as the comparator.  Returns the JSON line (printed when
    emit)."""
    import torch
    from paper_2504_03909_b300 import native, paillier as P

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    M, F, K, n_bits, depth = cfg["M"], cfg["F"], cfg["K"], cfg["n_bits"], cfg["depth"]
    L = n_bits // 32
    data_cfg = dict(cfg, seed=cfg.get("data_seed", cfg["seed"]))
    p, q, gh, r, bins = make_inputs(data_cfg)
    levels = synth.gen_tree_levels(M, depth, cfg["seed"])
    key = P.Key.from_primes(n_bits, p, q)
    if args.autotune:
        for op in (native.OP_ENCRYPT, native.OP_DECRYPT, native.OP_HIST):
            P.autotune(key, op, None)
    v = torch.from_numpy(gh.reshape(-1).copy()).to(dev)
    r_d = torch.from_numpy(r.view(np.int32)).to(dev)
    bins_d = torch.from_numpy(bins).to(dev)
    nodes_d = [torch.from_numpy(lv).to(dev) for lv in levels]
    node_buf = torch.empty(M, dtype=torch.int32, device=dev)
    maxn = 1 << (depth - 1)
    ct = torch.empty((2 * M, 2 * L), dtype=torch.int32, device=dev)
    ctm = torch.empty_like(ct)
    hist = torch.empty((maxn, F, K, 2, 2 * L), dtype=torch.int32, device=dev)
    cnt = torch.empty((maxn, F, K), dtype=torch.int32, device=dev)
    sums = torch.empty((maxn * F * K * 2,), dtype=torch.int64, device=dev)
    plan = P.LevelPlan(key, M, F, K, maxn)
    stream = torch.cuda.Stream()

    pack_bits = args.pack_bits
    B = args.gh_bits  # g/h packing: one plaintext enc(g) + 2^B enc(h) per sample (0: off)
    if B:
        # the histogram slot of a g/h cell holds S_g + 2^B S_h: 2B bits when packed
        pack_bits = 2 * B if args.pack_bits else 0
        hist_gh = torch.empty((maxn, F, K, 2 * L), dtype=torch.int32, device=dev)
        m2 = torch.empty((M, 2), dtype=torch.int64, device=dev)
        ct1 = torch.empty((M, 2 * L), dtype=torch.int32, device=dev)
        ctm1 = torch.empty_like(ct1)
    slots = P.pack_slots(key, pack_bits) if pack_bits else 0
    packed = (torch.empty((-(-(maxn * F * K * 2) // slots), 2 * L), dtype=torch.int32, device=dev)
              if pack_bits else None)
    split_nodes = torch.zeros(M, dtype=torch.int32, device=dev)

    level_slots = {}

    def cells_per_packed(nc):
        """Cells per packed ciphertext for a level of nc cells: each packed
        ciphertext is a serial chain of (slots - 1)(B + 1) products, so a level
        with few cells keeps at least 1,024 of them (the rule of the serving
        loop); --pack-slots caps it instead.  1: decrypt the cells directly."""
        if args.pack_slots:
            s_ = min(slots, args.pack_slots)
        else:
            s_ = min(slots, -(-nc // 1024))
        s_ = max(s_, -(-nc // packed.shape[0]))   # within the packed buffer
        level_slots[nc] = s_
        return s_

    def decrypt_level(nn):
        if B:
            cells = hist_gh[:nn].reshape(-1, 2 * L)
            nc = cells.shape[0]
            out = sums[:2 * nc].view(nc, 2)
            s_ = cells_per_packed(nc) if pack_bits else 1
            if s_ > 1:
                npk = -(-nc // s_)
                P.pack(key, cells, pack_bits, out=packed[:npk], slots=s_)
                P.decrypt_packed_gh(key, packed[:npk], nc, B, out=out, slots=s_)
            else:
                P.decrypt_gh(key, cells, B, out=out)
            return
        cells = hist[:nn].reshape(-1, 2 * L)
        nc = cells.shape[0]
        s_ = cells_per_packed(nc) if pack_bits else 1
        if s_ > 1:
            npk = -(-nc // s_)
            P.pack(key, cells, pack_bits, out=packed[:npk], slots=s_)
            P.decrypt_packed_u64(key, packed[:npk], nc, pack_bits, out=sums[:nc], slots=s_)
        else:
            P.decrypt_u64(key, cells, out=sums[:nc])

    plan_gh = P.LevelPlan(key, M, F, K, maxn, gh=True) if B else None

    def level_hist(nn):
        """This level's encrypted histograms of the nodes in node_buf (one
        captured graph per plan, replayed for every level)."""
        if B:
            plan_gh.run(ctm1, bins_d, node_buf, nn, hist=hist_gh, count=cnt)
        else:
            plan.run(ctm.view(2, M, 2 * L), bins_d, node_buf, nn, hist=hist, count=cnt)

    def tree_step(with_decrypt=True):
        if B:
            P.encode_gh(v[:M], v[M:], B, out=m2)
            P.encrypt_gh(key, m2, r_d[:M], out=ct1)
            P.ct_prepare(key, ct1, out=ctm1)
        else:
            m = P.encode(v)
            P.encrypt(key, m, r_d, out=ct)
            P.ct_prepare(key, ct, out=ctm)
        if args.splits == "data":
            split_nodes.zero_()
        parent = None
        for lvl in range(depth):
            nn = 1 << lvl
            if args.splits == "data":
                node_buf.copy_(split_nodes)
            else:
                node_buf.copy_(nodes_d[lvl])
            if parent is not None:
                # histogram subtraction: only the smaller child of each parent is aggregated and decrypted
                psums, pcnt, pf, pb = parent
                small_right, small_node = P.child_select(node_buf, pcnt, pf, pb)
                node_buf.copy_(small_node)
                level_hist(nn // 2)
                decrypt_level(nn // 2)
                lsums, lcnt = P.child_subtract(psums, pcnt, sums[:nn // 2 * F * K * 2].view(nn // 2, F, K, 2),
                                               cnt[:nn // 2], small_right)
                node_buf.copy_(split_nodes)
            else:
                level_hist(nn)
                if not with_decrypt:
                    continue
                decrypt_level(nn)
                lsums, lcnt = sums[:nn * F * K * 2].view(nn, F, K, 2), cnt[:nn]
            if args.splits == "data" and lvl + 1 < depth:
                bf, bb, _ = P.split_find(lsums, lcnt, 1.0, 0.0, 1.0)
                P.split_apply(bins_d, node_buf, bf, bb, out=split_nodes)
                if args.subtract:
                    parent = (lsums.clone(), lcnt.clone(), bf, bb)

    def hist_levels(per_node):
        for lvl in range(depth):
            nn = 1 << lvl
            if B:  # g/h packed: one ciphertext array, batched launches only
                node_buf.copy_(nodes_d[lvl])
                level_hist(nn)
            elif per_node:
                P.hist_aggregate(key, ctm.view(2, M, 2 * L), bins_d, nodes_d[lvl], nn, K, hist=hist[:nn],
                                 count=cnt[:nn], per_node=True)
            else:
                node_buf.copy_(nodes_d[lvl])
                plan.run(ctm.view(2, M, 2 * L), bins_d, node_buf, nn, hist=hist, count=cnt)

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            tree_step()
        P.sync(stream)
        with ClockSampler(local) as clk:
            native.call("paillier_profile", 1)
            t_tree = timed(tree_step, args.steps)
            prof = {}
            for kname in ("modexp_enc1", "modexp_enc", "enc_crt", "modexp_dec", "dec_crt", "to_mont", "pack", "unpack"):
                tot = native.C.c_double(0)
                cl = native.C.c_longlong(0)
                native.call("paillier_profile_read", kname.encode(), native.C.byref(tot), native.C.byref(cl))
                prof[kname] = tot.value / args.steps
            native.call("paillier_profile", 0)
            hist_levels(False)
            t_batched = timed(lambda: hist_levels(False), args.steps)
            t_per_node = None
            if not args.no_compare and not B:
                hist_levels(True)
                t_per_node = timed(lambda: hist_levels(True), args.steps)
        P.sync(stream)
        # untimed: the root histogram of this step's ciphertexts, decrypted, equals the plaintext sums
        node0 = torch.zeros(M, dtype=torch.int32, device=dev)
        if B:
            h0, c0 = P.hist_aggregate_gh(key, ctm1, bins_d, node0, 1, K)
            got = P.decrypt_gh(key, h0.reshape(-1, 2 * L), B)
        else:
            h0, c0 = P.hist_aggregate(key, ctm.view(2, M, 2 * L), bins_d, node0, 1, K)
            got = P.decrypt_u64(key, h0.reshape(-1, 2 * L))
        want, want_cnt = plaintext_root_sums(P, torch, v, bins_d, M, F, K)
        P.sync(stream)
        if not (torch.equal(got.view(F * K, 2), want) and torch.equal(c0.view(-1).long(), want_cnt)):
            raise RuntimeError("decrypted root histogram differs from the plaintext sums")
        del h0, c0, got, want, want_cnt
    ct_mults = 0
    strict = 0
    for lv in levels:
        inn = int((lv >= 0).sum())
        ct_mults += (1 if B else 2) * F * inn
    cells = sum((1 << lvl) * F * K * 2 for lvl in range(depth))
    line = {
        "metric": METRIC, "value": ct_mults / t_batched, "unit": "ct-mults/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tree, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{args.config}: depth-{depth} tree ({(1 << depth) - 1} nodes, "
                               + ("Beta(0.5,0.5) splits" if args.splits == "beta" else
                                  "splits found on the decrypted histograms")
                               + f") on {M:,} samples x {F} features x {K} bins, {n_bits}-bit n; step = encrypt "
                               "+ per-level histograms + CRT decrypt of every level's cells",
                   "M": M, "F": F, "K": K, "n_bits": n_bits,
                   "depth": depth, "autotuned": bool(args.autotune),
                   "configs": {op: P.get_config(key, i) for i, op in enumerate(("encrypt", "decrypt", "hist"))}},
        "hist_batched_ms_per_tree": 1e3 * t_batched,
        "hist_per_node_ms_per_tree": 1e3 * t_per_node if t_per_node else None,
        "batched_speedup_vs_per_node": t_per_node / t_batched if t_per_node else None,
        "ct_mults_per_tree": ct_mults,
        "tree_ms": 1e3 * t_tree,
        "phases_ms_per_tree": {"encrypt": prof["modexp_enc1"] + prof["modexp_enc"] + prof["enc_crt"],
                               "prepare": prof["to_mont"],
                               "pack": prof["pack"],
                               "decrypt": prof["modexp_dec"] + prof["dec_crt"] + prof["unpack"]},
        "decrypted_cells_per_tree": cells,
        "pack_bits": pack_bits, "pack_slots": slots,
        "pack_slots_by_level_cells": {str(k): v for k, v in sorted(level_slots.items())},
        "splits": args.splits, "subtract": bool(args.subtract),
        "gh_bits": B, "encryptions_per_tree": M if B else 2 * M,
        "cells_decoded_per_s": cells / ((prof["modexp_dec"] + prof["dec_crt"] + prof["unpack"] + prof["pack"]) * 1e-3),
        "graph": (plan_gh if B else plan).stats(),
        "clocks": clk.summary(),
        "verified": f"root histogram of the step's ciphertexts, decrypted, == plaintext sums of the encoded "
                    f"values, all {F * K * 2} cells and counts (untimed)",
    }
    if rank == 0 and emit:
        emit_json(line)
    return line


def run_serving(args, cfg, emit=True):
    """Four simulated passive parties send Poisson-arriving histogram + decrypt
    requests (M log-uniform in [1e3, 1e6], F uniform in [8, 64], K uniform on
    {64, 96, ..., 256}, 2048- or 3072-bit key with p = 0.5) to one server; the
    ciphertexts and bins stay resident.  Offered load = --load x the capacity
    measured with a closed loop first.  Reports p50/p99 latency and throughput."""
    import random as pyrandom
    import threading as th
    import torch
    from paper_2504_03909_b300 import native, paillier as P

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    MMAX, FMAX, NUNIQ = 1_000_000, 64, 65_536
    keys, ctms = {}, {}
    for n_bits, seed in ((2048, 41), (3072, 42)):
        p, q = synth.gen_primes(n_bits, seed)
        key = P.Key.from_primes(n_bits, p, q)
        L = n_bits // 32
        gh = synth.gen_gh(NUNIQ, seed)
        r = synth.gen_r(p * q, n_bits, 2 * NUNIQ, seed, p, q)
        if args.gh_bits:  # one g/h-packed ciphertext per sample
            g_d, h_d = torch.from_numpy(gh[0].copy()).to(dev), torch.from_numpy(gh[1].copy()).to(dev)
            ct = P.encrypt_gh(key, P.encode_gh(g_d, h_d, args.gh_bits), P.to_limb_tensor(r[:NUNIQ], dev))
            ct = ct.view(1, NUNIQ, 2 * L)
        else:
            m = P.encode(torch.from_numpy(gh.reshape(-1)).to(dev))
            ct = P.encrypt(key, m, P.to_limb_tensor(r, dev)).view(2, NUNIQ, 2 * L)
        # the resident dataset repeats the NUNIQ encrypted samples up to MMAX rows
        full = ct.repeat(1, (MMAX + NUNIQ - 1) // NUNIQ, 1)[:, :MMAX].contiguous()
        if args.gh_bits:
            full = full.view(MMAX, 2 * L)
        keys[n_bits] = key
        ctms[n_bits] = P.ct_prepare(key, full)
        del ct, full
    kgrid = list(range(64, 257, 32))
    gen = torch.Generator(device=dev)
    gen.manual_seed(4)
    bins = [{K: torch.randint(0, K, (FMAX, MMAX), generator=gen, device=dev, dtype=torch.uint8) for K in kgrid}
            for _ in range(4)]
    P.sync()
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.5)
    rng = pyrandom.Random(4)

    def draw():
        nb = 2048 if rng.random() < 0.5 else 3072
        M = int(round(10 ** rng.uniform(3, 6)))
        return dict(nb=nb, party=rng.randrange(4), M=M, F=rng.randint(8, 64), K=rng.choice(kgrid))

    def submit(srv, rq):
        return srv.submit(keys[rq["nb"]], ctms[rq["nb"]], rq["M"], rq["F"], rq["K"], bins[rq["party"]][rq["K"]],
                          gh_stride=MMAX, bins_stride=MMAX, pack_bits=args.pack_bits, gh_bits=args.gh_bits,
                          pack_slots=args.pack_slots)

    ngh = 1 if args.gh_bits else 2

    def work(rq):
        """Modelled multiply-adds of a request: its histogram products mod n^2 plus
        its decryptions (per packed ciphertext when packing)."""
        L = rq["nb"] // 32
        w = 6 if rq["nb"] >= 2048 else 5
        cells = ngh * rq["F"] * rq["K"]
        slot_bits = 2 * args.gh_bits if args.gh_bits else args.pack_bits
        # the cells per packed ciphertext the server chooses for this request
        slots = P.Server.request_plan(keys[rq["nb"]], rq["M"], rq["F"], rq["K"], pack_bits=args.pack_bits,
                                      gh_bits=args.gh_bits, pack_slots=args.pack_slots)[0]
        if slots:
            dec = -(-cells // slots) * dec_imad(rq["nb"], w) + cells * (slot_bits + 2) * mont_imad(2 * L)
        else:
            dec = cells * dec_imad(rq["nb"], w)
        return ngh * rq["M"] * rq["F"] * mont_imad(2 * L) + dec

    srv = P.Server(slots=args.slots, hbm_budget=budget, promote_ms=args.promote_ms, chunk_imad=args.chunk_imad)
    # warm-up, then the closed-loop capacity in work units (every slot busy)
    warm = [draw() for _ in range(max(4 * args.slots, 32))]
    for rq in warm[:args.slots]:
        t, _, _ = submit(srv, rq)
        srv.wait(t)
    t0 = time.perf_counter()
    tick = [submit(srv, rq)[0] for rq in warm]
    for t in tick:
        srv.wait(t)
    work_rate = sum(work(rq) for rq in warm) / (time.perf_counter() - t0)
    mean_work = float(np.mean([work(draw()) for _ in range(20000)]))
    capacity = work_rate / mean_work
    rate = args.load * capacity
    reqs = [draw() for _ in range(args.requests)]
    gaps = [rng.expovariate(rate) for _ in reqs]
    done_lat = []
    tickets = []
    with ClockSampler(0) as clk:
        t_start = time.perf_counter()
        t_next = t_start
        for rq, g in zip(reqs, gaps):
            t_next += g
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(submit(srv, rq)[0])
        done_rq = []
        for t, rq in zip(tickets, reqs):
            st, lat = srv.wait(t)
            if st == native.REQ_DONE:
                done_lat.append(lat)
                done_rq.append(rq)
            srv.release(t)
        wall = time.perf_counter() - t_start
    stats = srv.stats()
    srv.close()
    lat = np.array(done_lat)
    work_mults = sum(2 * rq["M"] * rq["F"] for rq in reqs)
    work_cells = sum(2 * rq["F"] * rq["K"] for rq in reqs)
    line = {
        "metric": METRIC, "value": float(np.percentile(lat, 50)), "unit": "ms (p50 request latency)", "n_gpus": 1,
        "steps": args.requests, "warmup": len(warm), "ms_per_step": 1e3 * wall / args.requests,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "serving: 4 passive parties, Poisson arrivals, histogram + CRT-decrypt requests, "
                               "M log-uniform [1e3, 1e6], F uniform [8, 64], K uniform {64..256 step 32}, "
                               "2048/3072-bit keys p = 0.5, resident ciphertexts", "slots": args.slots,
                   "hbm_budget_bytes": budget, "offered_load": args.load, "requests": args.requests,
                   "promote_ms": args.promote_ms, "chunk_imad": args.chunk_imad,
                   "pack_bits": args.pack_bits, "gh_bits": args.gh_bits,
                   "pack_slots": args.pack_slots or "auto"},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "by_size": serving_classes(done_rq, lat, work),
        "mean_ms": float(lat.mean()), "throughput_req_per_s": len(lat) / wall,
        "capacity_req_per_s": capacity, "arrival_rate_req_per_s": rate,
        "ct_mults_per_s": work_mults / wall, "decrypts_per_s": work_cells / wall,
        "server": stats, "clocks": clk.summary(),
    }
    if emit:
        emit_json(line)
    return line


def serving_classes(reqs, lat, work):
    """p50/p99 latency per request size class (thirds of the modelled work
    distribution's log range: small, medium, large), beside each class's
    median modelled work."""
    if not reqs:
        return {}
    wk = np.array([work(rq) for rq in reqs], dtype=np.float64)
    lw = np.log(wk)
    edges = np.quantile(lw, [1 / 3, 2 / 3])
    out = {}
    for name, sel in (("small", lw <= edges[0]), ("medium", (lw > edges[0]) & (lw <= edges[1])),
                      ("large", lw > edges[1])):
        if sel.any():
            out[name] = {"n": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50)),
                         "p99_ms": float(np.percentile(lat[sel], 99)),
                         "median_work_TIMAD": float(np.median(wk[sel])) / 1e12}
    return out


def run_legs(args, line):
    """The other two parts of the metric, measured after the level headline in
    the same run (one GPU): the batched depth-6 tree (one captured graph per
    level, autotuned launch configurations) against the plain per-node launch
    path, the same tree as the secure tree with the decrypt-count reductions,
    and the serving loop's p50/p99 request latency at offered load 0.7 (two
    ciphertext arrays, then one g/h-packed array)."""
    import torch
    torch.cuda.empty_cache()
    ba = argparse.Namespace(**vars(args))
    ba.config, ba.steps, ba.warmup, ba.autotune = "batched", 2, 1, True
    ba.gh_bits, ba.pack_bits, ba.splits, ba.subtract, ba.no_compare = 0, 0, "beta", False, False
    b = run_batched(ba, synth.CONFIGS["batched"], emit=False)
    line["batched"] = {
        "workload": b["config"]["workload"], "autotuned": b["config"]["autotuned"],
        "configs": b["config"]["configs"],
        "hist_batched_ms_per_tree": b["hist_batched_ms_per_tree"],
        "hist_per_node_ms_per_tree": b["hist_per_node_ms_per_tree"],
        "speedup_vs_per_node": b["batched_speedup_vs_per_node"],
        "ct_mults_per_s_batched": b["value"], "tree_ms": b["tree_ms"], "phases_ms_per_tree": b["phases_ms_per_tree"],
        "steps": ba.steps, "warmup": ba.warmup, "clocks": b["clocks"], "verified": b["verified"],
    }
    torch.cuda.empty_cache()
    # the secure tree with the decrypt-count reductions: splits found on the
    # decrypted histograms, histogram subtraction, g/h packing (B = 45) and
    # ciphertext packing in 90-bit slots
    st = argparse.Namespace(**vars(ba))
    st.gh_bits, st.pack_bits, st.splits, st.subtract, st.no_compare = 45, 45, "data", True, True
    t = run_batched(st, synth.CONFIGS["batched"], emit=False)
    line["secure_tree"] = {
        "workload": t["config"]["workload"], "gh_bits": t["gh_bits"], "slot_bits": t["pack_bits"],
        "pack_slots": t["pack_slots"], "pack_slots_by_level_cells": t["pack_slots_by_level_cells"],
        "splits": t["splits"], "subtract": t["subtract"],
        "encryptions_per_tree": t["encryptions_per_tree"], "tree_ms": t["tree_ms"],
        "phases_ms_per_tree": t["phases_ms_per_tree"], "ct_mults_per_s_batched": t["value"],
        "steps": st.steps, "warmup": st.warmup, "clocks": t["clocks"], "verified": t["verified"],
    }
    torch.cuda.empty_cache()
    sa = argparse.Namespace(**vars(args))
    sa.config, sa.requests, sa.load, sa.slots = "serving", args.serve_requests, 0.7, 8
    sa.gh_bits, sa.pack_bits = args.serve_gh_bits, args.serve_pack_bits
    sv = run_serving(sa, synth.CONFIGS.get("serving", {}), emit=False)
    line["serving"] = {
        "workload": sv["config"]["workload"], "offered_load": sa.load, "requests": sa.requests, "slots": sa.slots,
        "gh_bits": sa.gh_bits, "pack_bits": sa.pack_bits, "pack_slots": sa.pack_slots or "auto",
        "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "mean_ms": sv["mean_ms"], "by_size": sv["by_size"],
        "throughput_req_per_s": sv["throughput_req_per_s"], "capacity_req_per_s": sv["capacity_req_per_s"],
        "server": sv["server"], "clocks": sv["clocks"],
    }
    # the same serving workload over one g/h-packed ciphertext per sample (half
    # the histogram products and decryptions; 90-bit packing slots)
    torch.cuda.empty_cache()
    sg = argparse.Namespace(**vars(sa))
    sg.gh_bits, sg.pack_bits = 45, 46
    sv = run_serving(sg, synth.CONFIGS.get("serving", {}), emit=False)
    line["serving_gh"] = {
        "gh_bits": sg.gh_bits, "pack_bits": sg.pack_bits, "pack_slots": sg.pack_slots or "auto",
        "offered_load": sg.load, "requests": sg.requests, "slots": sg.slots,
        "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "mean_ms": sv["mean_ms"], "by_size": sv["by_size"],
        "throughput_req_per_s": sv["throughput_req_per_s"], "capacity_req_per_s": sv["capacity_req_per_s"],
        "clocks": sv["clocks"],
    }


# The result line goes to the process's original standard output; everything
# else (libraries that print banners, e.g. NCCL's version line) goes to stderr.
_JSON_OUT = None


def reserve_stdout():
    """Keeps a private handle on standard output for the JSON line and points
    file descriptor 1 at stderr for the rest of the process."""
    global _JSON_OUT
    if _JSON_OUT is None:
        sys.stdout.flush()
        _JSON_OUT = os.fdopen(os.dup(1), "w")
        os.dup2(2, 1)


def emit_json(obj):
    out = _JSON_OUT if _JSON_OUT is not None else sys.stdout
    out.write(json.dumps(obj) + "\n")
    out.flush()


def main():
    reserve_stdout()
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="level",
                    choices=["level", "toy", "level_small", "batched", "serving", "large", "horizontal", "oracle"])
    ap.add_argument("--requests", type=int, default=300, help="serving: timed requests")
    ap.add_argument("--slots", type=int, default=8, help="serving: concurrent request slots")
    ap.add_argument("--load", type=float, default=0.7, help="serving: offered load / measured capacity")
    ap.add_argument("--promote-ms", type=float, default=None,
                    help="serving: aging threshold of large requests (the library's default when omitted)")
    ap.add_argument("--autotune", action="store_true", help="autotune the launch configurations first (batched)")
    ap.add_argument("--no-compare", action="store_true", help="batched/large: skip the per-node comparator")
    ap.add_argument("--pack-bits", type=int, default=0, help="batched/large: pack cells into B-bit slots before decryption")
    ap.add_argument("--subtract", action="store_true", help="tree modes with --splits data: histogram subtraction")
    ap.add_argument("--splits", default="beta", choices=["beta", "data"],
                    help="batched/large: Beta(0.5,0.5) splits or splits found on the decrypted histograms")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nodes", type=int, default=1, help="horizontal: node histograms per round")
    ap.add_argument("--gh-bits", type=int, default=None,
                    help="g/h packing, one plaintext enc(g) + 2^B enc(h) per sample (B bits; 0 = off): tree and "
                         "serving modes use it instead of two ciphertexts per sample; the level mode reports it "
                         "beside the headline (default 45 there, 0 elsewhere)")
    ap.add_argument("--shard", action="store_true",
                    help="level: run the sharded job (the N > 1 path) even on one rank")
    ap.add_argument("--no-legs", action="store_true",
                    help="level: skip the batched-tree and serving legs measured after the headline")
    ap.add_argument("--serve-requests", type=int, default=300, help="serving leg of the level run: timed requests")
    ap.add_argument("--serve-gh-bits", type=int, default=0, help="serving leg: g/h packing bits (0 = two arrays)")
    ap.add_argument("--serve-pack-bits", type=int, default=46, help="serving leg: ciphertext packing bits")
    ap.add_argument("--chunk-imad", type=float, default=None,
                    help="serving: modelled multiply-adds per launch (the library's default when omitted)")
    ap.add_argument("--pack-slots", type=int, default=0,
                    help="serving and tree modes: cells per packed ciphertext at most (0 = the rule: at least "
                         "1,024 packed ciphertexts for a request of little histogram work or a tree level; a "
                         "large value = as many as fit)")
    args = ap.parse_args()
    cfg = synth.CONFIGS.get(args.config, {})
    if args.gh_bits is None:
        args.gh_bits = 45 if args.config == "level" else 0
    if args.config == "oracle":
        run_oracle_rates(args)
    elif args.impl == "reference" and args.config == "horizontal":
        run_reference_horizontal(args, cfg)
    elif args.impl == "reference":
        run_reference(args, cfg)
    elif args.config == "horizontal":
        run_horizontal(args, cfg)
    elif args.config == "batched":
        run_batched(args, cfg)
    elif args.config == "serving":
        run_serving(args, cfg)
    elif args.config == "large":
        run_batched(args, cfg)
    elif (int(os.environ.get("WORLD_SIZE", "1")) > 1 or args.shard) and args.config == "level":
        run_sharded(args, cfg)
    else:
        line = run_ours(args, cfg)
        if line is not None:
            if args.gpus == 1 and not args.no_legs and args.config == "level":
                try:
                    run_legs(args, line)
                except Exception as exc:  # a failed leg must not cost the headline line
                    import traceback
                    traceback.print_exc()
                    line["legs_error"] = f"{type(exc).__name__}: {exc}"
            emit_json(line)


if __name__ == "__main__":
    main()
