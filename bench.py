"""Benchmark of the NSHEDB equality predicate on B300 (libhp).

Workload (default, --config plain): n = 2^26 slots = 2048 BFV ciphertext
pairs at N = 32768, L = 15 (log QP = 881), p = 65537; plaintext columns are
16-bit integers with y = x in half the slots (synthetic stand-in for the
paper's TPC-H columns).  One step = one pass of the whole hot path over the
batch: difference, 16 squarings with relinearisation, "1 -".

Prints one JSON line (rank 0).  value = slots compared per second over all
ranks (elements/s), device-resident inputs.  e2e = the same metric through
hp_run with pinned host buffers (copies inside the timed region).
`--impl reference` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import queue
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_24271_b300.sharding import allgather_partials, max_over_ranks, rank_seed  # noqa: E402

METRIC = "hot-path elements/s and % roofline, batched vs plain at stated error, 1 B300"
UNIT = "elements/s"
LOGN = 15
SEED_KEY, SEED_DATA = 1, 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libhp", choices=["libhp", "reference"])
    ap.add_argument("--config", default="plain", choices=["plain", "const28", "batched", "lt", "between", "in", "sum", "rotsum", "join"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--n-ct", type=int, default=0, help="override the ciphertext count (diagnostics only)")
    ap.add_argument("--ks-digit-primes", type=int, default=0, choices=[0, 3, 5],
                    help="data primes per key-switching digit (0: the workload's default)")
    ap.add_argument("--ks-fine-depth", type=int, default=-1,
                    help="depth up to which per-prime digits relinearise (-1: the workload's default)")
    ap.add_argument("--ks-coarse-from", type=int, default=-1,
                    help="depth from which the two-digit key relinearises (0: never; -1: the workload's default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="default line: skip the batched-vs-plain comparison")
    ap.add_argument("--no-extras", action="store_true", help="default line: skip the 2^28-slot and reduced-size row extras")
    ap.add_argument("--ncu-region", action="store_true",
                    help="after warm-up, run one extra step between cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


def workload(cfg: str):
    if cfg == "between":
        return dict(n_ct=64, op="between", desc="x BETWEEN 1000 AND 20000 (Sec. 4.2.2: (1 - LT(x, lo)) (1 - LT(hi, x))): "
                    "2^21 slots = 64 BFV ciphertexts, x in [0, 2^15], N=32768, L=15, p=65537; two LT evaluations "
                    "and their product (1023 multiplications) per ciphertext, bit-exact")
    if cfg == "join":
        return dict(n_ct=64, op="join", n_rows=16, desc="equi-join A.key = B.key (Sec. 4.2.2, Extract + Broadcast): "
                    "A = 2^21 rows (64 BFV ciphertexts), 16 B rows with 2 attributes; 1024 EQ chains, 2048 products, "
                    "48 broadcasts per step; N=32768, L=15, p=65537, bit-exact; value = A-row x B-row comparisons/s")
    if cfg == "sum":
        return dict(n_ct=2048, op="sum", desc="SUM(y) WHERE x = c: SELECT (Eq. 5: EQ chain + column x mask) over 2^26 "
                    "slots = 2048 BFV ciphertext pairs, then the whole column reduced by the rotate-and-add "
                    "reduction (Sec. 4.2.2) into one ciphertext; N=32768, L=15, p=65537, bit-exact; value = slots/s")
    if cfg == "rotsum":
        return dict(n_ct=512, op="rotsum", desc="rotate-and-add reduction (COUNT/SUM, Sec. 4.2.2) of each of 512 BFV "
                    "ciphertexts (2^24 slots): 15 rotations with key switching per ciphertext, N=32768, L=15, "
                    "p=65537, bit-exact; value = slots reduced/s")
    if cfg == "in":
        return dict(n_ct=256, op="in", n_const=8,
                    desc="IN(x, S) (Eq. 6) with |S| = 8 constants, GROUP BY fan-out of 8 EQ chains per ciphertext: "
                    "2^23 slots = 256 BFV ciphertexts, N=32768, L=15, p=65537, bit-exact; value = slot-constant "
                    "comparisons/s")
    if cfg == "lt":
        return dict(n_ct=64, op="lt", desc="LT(x, y) = [x < y] (Eq. 4): 2^21 slots = 64 BFV ciphertext pairs, "
                    "x, y in [0, 2^15], N=32768, L=15, p=65537; 511 multiplications per ciphertext, bit-exact")
    if cfg == "batched":
        return dict(n_ct=0, op="batched", desc="batched EQ(x, y): 4096 instances, sizes log-uniform in [2^8, 2^16] slots, "
                    "dictionary IDs in [1, 2^15], N=32768, L=15, p=65537, bit-exact; slot-packed into shared ciphertexts")
    if cfg == "const28":
        return dict(n_ct=8192, op="const", desc="EQ(x, c): 2^28 slots = 8192 BFV ciphertexts vs a broadcast constant, "
                    "N=32768, L=15 (log QP=881), p=65537, bit-exact")
    return dict(n_ct=2048, op="ctct", desc="EQ(x, y): 2^26 slots = 2048 BFV ciphertext pairs, N=32768, L=15 "
                "(log QP=881), p=65537, 16 squarings + relinearisation, bit-exact")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------
NTT_CLASSES = {0, 1, 2, 3}
# per unit, in multiplier lane-slots: a butterfly's Shoup product is 9 single-slot
# multiplies (3 wide, 2 high, 4 low); a 64-bit multiply-accumulate is 4 wide
# multiply-adds with a 64-bit addend, two slots each (the ratio of the two
# register-only probes, 0.97 T butterflies/s and 1.06 T MAC/s, agrees)
N_SM, MUL_LANES_PER_SM_CLK, MUL_PER_BUTTERFLY, MUL_PER_MAC = 148, 32, 9, 8
MAC_PER_UNIT = {4: 15 * 16, 6: 2 * 15 * 16, 8: 1}  # lift, scale-and-round, key-switch MAC
# ciphertext multiplications with relinearisation per N units of each workload
# (per ciphertext; per ciphertext and B row for join); rotations are not counted
HMULT_PER_CT = {"ctct": 16, "const": 16, "in": 16, "lt": 511, "between": 1023, "sum": 17, "rotsum": 0, "join": 18}
# Shoup products of the digit recombination per ciphertext and multiplication, in
# units of N, for digits of G primes: per digit (15 / G) and target prime outside
# the digit's own primes, G - 1 products (a digit's value modulo one of its own
# primes is d2's residue, read as stored): G = 3: 5 x 13 x 2 = 130; G = 5:
# 3 x 11 x 4 = 132; the two-digit key (8 and 7 primes): 8 x 7 + 9 x 6 = 110
DIGIT_PRODUCTS_PER_HMULT = {3: 130, 5: 132, 8: 110}
TC_FLOPS_PER_COEFF = 2 * 128 * 128  # one tensor-core conversion MMA, per coefficient
# key switching per workload: (per-prime digits up to this depth, data primes
# per digit, depth from which the two-digit key relinearises).  The workloads
# built on EQ chains and rotations: five-prime digits (3 digits), whose depth-16
# chain keeps about 114 bits of noise budget with them at N = 32768 (enough for
# a product and a reduction after it), and the two-digit key from depth 7, where
# it no longer costs budget.  LT and BETWEEN: per-prime digits for their 8
# products up to depth 4 (the first levels, where key-switching noise costs
# budget), five-prime digits for depths 5 .. 9, the two-digit key from depth 10
DEFAULT_KEY_SWITCHING = {"ctct": (0, 5, 7), "const": (0, 5, 7), "batched": (0, 5, 7), "in": (0, 5, 7),
                         "sum": (0, 5, 7), "rotsum": (0, 5, 7), "join": (0, 5, 7), "lt": (4, 5, 10),
                         "between": (4, 5, 10)}


def fine_depth(args, op):
    return DEFAULT_KEY_SWITCHING[op][0] if args.ks_fine_depth < 0 else args.ks_fine_depth


def digit_primes(args, op):
    return args.ks_digit_primes or DEFAULT_KEY_SWITCHING[op][1]


def coarse_from(args, op):
    return DEFAULT_KEY_SWITCHING[op][2] if args.ks_coarse_from < 0 else args.ks_coarse_from


KERNEL_SOURCES = {  # files whose text determines a kernel's code
    "ntt": ["hp_defs.h", "hp_device.cuh", "hp_ntt.cuh"],
    "tc": ["hp_defs.h", "hp_device.cuh", "hp_rns.cuh", "hp_tc.cuh", "hp_tcconv.cuh"],
    "rns": ["hp_defs.h", "hp_device.cuh", "hp_rns.cuh"],
}


def source_hash(kernel: str) -> str:
    group = "ntt" if kernel.startswith("k_ntt") else ("tc" if kernel.endswith("_tc") else "rns")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[group]:
        h.update(open(os.path.join(ROOT, "paper_2602_24271_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str, tile: int):
    """dram bytes per launch for `kernel` from the committed ncu counter summary,
    scaled from the summary's tile to `tile` ciphertexts per launch (a transform
    launch's traffic is proportional to its polynomials), or None if the summary
    is missing or was taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_counters.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k or k.get("source_hash") != source_hash(kernel) or not d.get("tile_ct"):
        return None
    return k.get("dram_bytes_per_launch_full") * tile / d["tile_ct"]


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
def _ceil_log2(i: int) -> int:
    return (i - 1).bit_length()


def lt_product_depths():
    """Multiplicative depths of LT's 511 products (Eq. 4, the depth-optimal
    baby-step / giant-step schedule): w = z^2 at 1, baby powers w^i at
    1 + ceil(log2 i), giant powers w^(256 j) at 9 + ceil(log2 j), the giant-step
    products at 10 + ceil(log2 j), the final product with z at 18."""
    d = [1] + [1 + _ceil_log2(i) for i in range(2, 256)] + [9] + [9 + _ceil_log2(j) for j in range(2, 129)]
    return d + [10 + _ceil_log2(j) for j in range(1, 128)] + [18]


def product_depths(op: str):
    """Multiplicative depths of the multiplications one unit of a workload performs."""
    eq = list(range(1, 17))
    return {"ctct": eq, "const": eq, "batched": eq, "in": eq, "sum": eq + [17], "join": eq + [17, 17],
            "rotsum": [], "lt": lt_product_depths(), "between": 2 * lt_product_depths() + [19]}[op]


class OracleSample:
    """One ciphertext of the workload (N = 32768) on the CPU oracle, keys and
    encryptions made once, with the workload's key switching.  `time(n_mul)`
    times the oracle's primitives on it single-threaded (difference, `n_mul`
    multiplications with relinearisation by each key the workload uses, "1 -",
    and one rotation with key switching where the workload rotates) and composes
    the time of one unit of the workload from the counts below and the depths of
    its multiplications (product_depths: those at depth coarse_from or more are
    relinearised with the two-digit key).  The composition counts the
    multiplications and rotations the workload performs and the difference and
    "1 -" of each EQ chain; ciphertext additions, the plaintext products of
    Extract and LT's inner sums (255 scalar products per giant step) are left
    out, so for those workloads the rate is an upper bound on the oracle's."""

    # per ciphertext (per ciphertext and B row for join): (differences, "1 -",
    # rotations, what is left out)
    COUNTS = {
        "ctct": (1, 1, 0, ""),
        "const": (1, 1, 0, ""),
        "batched": (1, 1, 0, ""),
        "in": (1, 1, 0, "the additions of the IN sum"),
        "lt": (1, 0, 0, "the 128 inner sums of 255 scalar products and the additions"),
        "between": (3, 2, 0, "the 2 x 128 inner sums of 255 scalar products and the additions"),
        "sum": (1, 1, 15 / 2048, "the additions"),
        "rotsum": (0, 0, 15, "the additions"),
        "join": (1, 1, 45 / 64, "the plaintext products of Extract and the additions"),
    }

    def __init__(self, op: str = "ctct", dp: int = 3, coarse_from: int = 0, fine_depth: int = 0):
        import oracle
        from paper_2602_24271_b300.inputs import eq_pair_columns

        self.op, self.coarse_from, self.fine_depth = op, coarse_from, fine_depth
        self.o = oracle.Oracle(LOGN, dp=dp, coarse_from=coarse_from, fine_depth=fine_depth)
        self.o.keygen(SEED_KEY)
        x, y = eq_pair_columns(self.o.N, seed=SEED_DATA)
        self.cx, self.cy = self.o.encrypt(x, 7, 0), self.o.encrypt(y, 7, 1)
        self.g = None
        if self.COUNTS[op][2]:
            self.g = self.o.galois_elements()[0]
            self.o.galois_keygen(SEED_KEY, self.g)

    def time(self, n_mul: int = 1):
        o = self.o
        n_sub, n_1m, n_rot, left_out = self.COUNTS[self.op]
        depths = product_depths(self.op)
        cf, F = self.coarse_from, self.fine_depth
        n_fine = sum(1 for d in depths if d <= F)
        n_coarse = sum(1 for d in depths if d > F and cf and d >= cf)
        n_main = len(depths) - n_fine - n_coarse
        # (operand depth, count timed, count in the unit) per key: the per-prime
        # key relinearises a product of fresh operands (F > 0), the main key one
        # at depth F + 1, the two-digit key one at depth cf
        keys = [(0, n_mul if n_fine else 0, n_fine), (F, n_mul if n_main else 0, n_main),
                (cf - 1, n_mul if n_coarse else 0, n_coarse)]
        t0 = time.perf_counter()
        d = o.sub(self.cx, self.cy)
        t1 = time.perf_counter()
        t_mults = 0.0
        for depth_a, n_timed, n_unit in keys:
            if not n_timed:
                continue
            ta = time.perf_counter()
            for _ in range(n_timed):
                o.mul_relin(d, d, depth_a=depth_a, depth_b=depth_a)
            t_mults += n_unit * (time.perf_counter() - ta) / n_timed
        t2 = time.perf_counter()
        o.one_minus(d)
        t3 = time.perf_counter()
        t_rot = 0.0
        if self.g is not None:
            o.rotate(d, self.g)
            t_rot = time.perf_counter() - t3
        per_unit = n_sub * (t1 - t0) + t_mults + n_1m * (t3 - t2) + n_rot * t_rot
        desc = ("1 ciphertext at N=32768 (32768 slots) on the oracle, single-threaded, key-switching digits of %d "
                "primes%s%s: a difference, %d multiplication(s) with relinearisation per key used, '1 -'%s timed; "
                "one unit of the workload composed as %d difference(s) + %d multiplications (%d with the per-prime "
                "key, %d with the two-digit key) + %d x '1 -'%s%s" % (
                    o.dp, ", per-prime digits up to depth %d" % F if F else "",
                    ", the two-digit key from depth %d" % cf if cf else "", n_mul,
                    " and one rotation" if self.g is not None else "", n_sub, len(depths), n_fine, n_coarse, n_1m,
                    " + %.3g rotations" % n_rot if n_rot else "",
                    "; not counted: %s (the rate is an upper bound)" % left_out if left_out else ""))
        return o.N / per_unit, time.perf_counter() - t0, desc


def _oracle_worker(op, n_mul, barrier, results, dp, cf, F):
    sample = OracleSample(op, dp, cf, F)
    barrier.wait(timeout=120)  # every worker set up: the timed samples run concurrently
    results.put(sample.time(n_mul))


def multicore_baseline(op: str, n_mul: int = 1, max_workers: int = 32, dp: int = 3, cf: int = 0, F: int = 0):
    """The paper's multi-threaded form (Sec. 5.3: independent predicates
    assigned to threads): W = min(32, host cores) single-threaded oracle
    processes (about 0.45 GB of host memory each), started with spawn, set up
    (keys and one ciphertext each), released together by a barrier, then each
    times the cpu_baseline composition of one unit on its own ciphertext.  All
    W run at the same time, so the aggregate rate is the sum of their rates."""
    import multiprocessing as mp

    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    w = max(1, min(max_workers, cores))
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(w), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(op, n_mul, barrier, results, dp, cf, F)) for _ in range(w)]
    for pr in procs:
        pr.start()
    got, deadline = [], time.time() + 300
    while len(got) < w:
        try:
            got.append(results.get(timeout=2))
        except queue.Empty:
            if time.time() > deadline or not any(pr.is_alive() for pr in procs):
                break
    for pr in procs:
        pr.join(timeout=10)
        if pr.is_alive():
            pr.terminate()
    if len(got) < w:
        raise RuntimeError("%d of %d oracle worker processes reported" % (len(got), w))
    value = sum(v for v, _, _ in got)
    return {"value": value, "unit": UNIT, "cores": w, "host_cores": cores, "kind": "oracle",
            "sample": "%d concurrent single-threaded oracle processes (independent predicates on separate cores, "
                      "as in the paper's multi-threaded runs), released together; value = sum of their rates; "
                      "each: %s" % (w, got[0][2])}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.config)
    sample = OracleSample(wl["op"], digit_primes(args, wl["op"]), coarse_from(args, wl["op"]), fine_depth(args, wl["op"]))
    vals, step_ms, desc = [], [], ""
    for i in range(args.warmup + args.steps):
        v, secs, desc = sample.time(1)
        if i >= args.warmup:
            vals.append(v)
            step_ms.append(secs * 1e3)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl["desc"], "step": "one bounded sample of the workload (see cpu_baseline)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_libhp(args):
    import numpy as np
    import torch

    from paper_2602_24271_b300 import hp
    from paper_2602_24271_b300.inputs import eq_pair_columns
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = workload(args.config)
    n_ct = args.n_ct or wl["n_ct"]
    ctx = hp.Context(LOGN, max_tile_ct=args.tile, ks_digit_primes=digit_primes(args, wl["op"]),
                     ks_coarse_from=coarse_from(args, wl["op"]), ks_fine_depth=fine_depth(args, wl["op"]))
    ctx.keygen(SEED_KEY)
    if not args.ncu_region:
        ctx.autotune()
    N = ctx.N
    # inputs: rank r encrypts its own share (weak scaling, no exchange)
    x, y = eq_pair_columns(n_ct * N, seed=rank_seed(SEED_DATA, rank),
                           value_bits=15 if wl["op"] in ("lt", "between") else 16)
    const_val = 4242
    if wl["op"] == "sum":  # WHERE x = c holds in about a quarter of the rows; y is the summed column
        x[np.random.default_rng(rank_seed(SEED_DATA + 1, rank)).random(n_ct * N) < 0.25] = const_val
    if wl["op"] in ("sum", "rotsum", "join"):
        ctx.galois_keygen(SEED_KEY)
    if wl["op"] == "join":  # B: 16 rows with distinct keys drawn from A's column, two attribute columns
        jr = wl["n_rows"]
        bkey = np.zeros(N, dtype=np.uint32)
        bkey[:jr] = np.unique(x[: 64 * jr])[:jr]
        battr = np.random.default_rng(rank_seed(SEED_DATA + 2, rank)).integers(0, 65537, (2, N)).astype(np.uint32)
        cbk = ctx.encrypt(bkey.reshape(1, N), seed=SEED_DATA + 5, ct_index0=0)
        cba = [ctx.encrypt(battr[k].reshape(1, N), seed=SEED_DATA + 5, ct_index0=1 + k) for k in range(2)]
        jout = torch.empty((2, n_ct, 2, 15, N), dtype=torch.int64, device="cuda")
    cx = ctx.ct_empty(n_ct)
    cy = ctx.ct_empty(n_ct) if wl["op"] in ("ctct", "lt", "sum") else None
    chunk = 128
    for c0 in range(0, n_ct, chunk):
        c1 = min(n_ct, c0 + chunk)
        cx[c0:c1] = ctx.encrypt(x[c0 * N:c1 * N].reshape(-1, N), seed=SEED_DATA, ct_index0=c0)
        if cy is not None:
            cy[c0:c1] = ctx.encrypt(y[c0 * N:c1 * N].reshape(-1, N), seed=SEED_DATA, ct_index0=n_ct + c0)
    out = ctx.ct_empty(n_ct)
    agg = ctx.ct_empty(1)
    total_ct = ctx.ct_empty(1)
    in_consts = [int(v) for v in x[:wl.get("n_const", 0)]]  # members drawn from the column itself
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def step():
        if wl["op"] == "lt":
            ctx.run(hp.HP_LT, cx, cy, 0, out=out, stream=stream)
        elif wl["op"] == "in":
            ctx.eq_fanout(cx, in_consts, masks=False, in_set=out, stream=stream)
        elif wl["op"] == "between":
            ctx.between(cx, 1000, 20000, out=out, stream=stream)
        elif wl["op"] == "sum":
            ctx.run(hp.HP_SELECT, cx, cy, const_val, out=out, stream=stream)
            n = ctx.launch_count()
            ctx.rotate_sum(out, group=n_ct, out=agg, stream=stream)
            n += ctx.launch_count()
            if dist:  # the one exchange: all-gather the partial aggregates, add them mod Q
                ctx.ct_sum(allgather_partials(agg[0], dist), group=world, out=total_ct, stream=stream)
                n += ctx.launch_count()
            return n
        elif wl["op"] == "rotsum":
            ctx.rotate_sum(cx, out=out, stream=stream)
        elif wl["op"] == "join":
            ctx.join(cx, cbk, cba, wl["n_rows"], out=jout, stream=stream)
        elif cy is not None:
            ctx.run(hp.HP_EQ_CT_CT, cx, cy, 0, out=out, stream=stream)
        else:
            ctx.run(hp.HP_EQ_CT_CONST, cx, None, const_val, out=out, stream=stream)
        return ctx.launch_count()

    # one profiled warm-up step over every kernel class: shares and the dominant kernel
    ctx.profile((1 << len(hp.PROFILE_CLASSES)) - 1)
    step()
    shares, works = {}, {}
    for c, name in enumerate(hp.PROFILE_CLASSES):
        ms, n, w = ctx.profile_read(c)
        shares[c], works[c] = ms, w
    ctx.profile(0)
    dom = max(shares, key=shares.get)
    tot = sum(shares.values())
    for _ in range(max(0, args.warmup - 1)):
        step()
    torch.cuda.synchronize()

    if args.ncu_region:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()

    # ---- timed region ----
    ctx.profile(1 << dom)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        launches += step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    dom_ms, dom_n, dom_work = ctx.profile_read(dom)
    ctx.profile(0)
    ctx.check_status()
    ms_max = max_over_ranks(ms_total, dist, device="cuda")
    ms_per_step = ms_max / args.steps
    slots_all = n_ct * N * world * wl.get("n_const", 1) * wl.get("n_rows", 1)
    value = slots_all / (ms_per_step / 1e3)

    # correctness of this run (decrypt a few ciphertexts, closed form)
    probe = [0, n_ct // 2, n_ct - 1]
    dec = ctx.decrypt((jout[1] if wl["op"] == "join" else out)[probe])
    if wl["op"] == "sum":
        total = int(y[x == const_val].astype(np.int64).sum() % 65537)
        assert np.all(ctx.decrypt(agg) == total), "SUM result wrong in benchmark run"
        if dist:
            t = torch.tensor([total], dtype=torch.int64, device="cuda")
            dist.all_reduce(t)
            assert np.all(ctx.decrypt(total_ct) == int(t.item()) % 65537), "combined SUM wrong in benchmark run"
    for k, c in enumerate(probe):
        xs = x[c * N:(c + 1) * N]
        if wl["op"] == "sum":
            ref = np.where(xs == const_val, y[c * N:(c + 1) * N], 0)
        elif wl["op"] == "rotsum":
            ref = np.full(N, int(xs.astype(np.int64).sum() % 65537))
        elif wl["op"] == "join":
            ref = np.zeros(N, dtype=np.uint32)
            for r in range(wl["n_rows"]):
                ref[xs == bkey[r]] = battr[1][r]
        elif wl["op"] == "lt":
            ref = xs < y[c * N:(c + 1) * N]
        elif wl["op"] == "in":
            ref = np.isin(xs, in_consts)
        elif wl["op"] == "between":
            ref = (xs >= 1000) & (xs <= 20000)
        else:
            ref = (xs == y[c * N:(c + 1) * N]) if cy is not None else (xs == const_val)
        assert np.array_equal(dec[k], ref.astype(np.uint32)), "EQ result wrong in benchmark run"

    # ---- roofline of the dominant kernel ----
    avg_ms = dom_ms / max(1, dom_n)
    work_per_launch = dom_work / max(1, dom_n)
    kernel = hp.KERNEL_OF_CLASS[dom]
    # ALU peak from unit counts and the clock seen in the timed region: 148 SMs x
    # SM clock x 32 multiplier lane-slots per SM per clock (the FMA-heavy pipe),
    # / 9 slots per butterfly or / 8 per 64-bit multiply-accumulate
    mhz = clk.get("sm_mhz") or 2032.0
    mul_rate = N_SM * mhz * 1e6 * MUL_LANES_PER_SM_CLK
    if dom in NTT_CLASSES:
        peak, probe = mul_rate / MUL_PER_BUTTERFLY, hp.probe_peak(0)
        achieved = work_per_launch / (avg_ms / 1e3)
        roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gbutterfly/s"}
    elif dom in MAC_PER_UNIT:
        peak, probe = mul_rate / MUL_PER_MAC, hp.probe_peak(1)
        achieved = work_per_launch * MAC_PER_UNIT[dom] / (avg_ms / 1e3)
        roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "GMAC/s"}
    else:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        probe = None
        achieved = work_per_launch * 8 * 2 / (avg_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = kernel
    roof["launches_timed"] = dom_n
    roof["avg_launch_ms"] = avg_ms
    roof["share_of_step"] = shares[dom] / tot if tot else None
    if probe is not None:
        roof["peak_source"] = ("derived: 148 SMs x %.0f MHz x 32 multiplier lane-slots per SM per clock / %d slots "
                               "per unit" % (mhz, MUL_PER_BUTTERFLY if dom in NTT_CLASSES else MUL_PER_MAC))
        roof["probe_peak"] = probe / 1e9
        roof["frac_of_probe"] = roof["achieved"] / roof["probe_peak"]
    else:
        roof["peak_source"] = "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
    roof["probe_butterfly_per_s"] = hp.probe_peak(0)
    roof["probe_mac_per_s"] = hp.probe_peak(1)
    # the same butterfly on 32-bit words (a 30-bit prime), and modulus bits per
    # second through each: 55-bit primes here against 30-bit ones
    roof["probe_butterfly32_per_s"] = hp.probe_peak(2)
    roof["probe_modulus_bits_per_s"] = {"u64_55bit": 55 * roof["probe_butterfly_per_s"],
                                        "u32_30bit": 30 * roof["probe_butterfly32_per_s"]}
    roof["traffic"] = load_traffic(kernel, ctx_tile(ctx))
    # whole path: the step's algorithmic butterflies (every transform), digit
    # recombination products (counted at the butterfly rate) and key-switching
    # multiply-accumulates at the derived ALU ceilings, against the step time;
    # the base conversions run on the tensor cores and are not counted
    butterflies = sum(works[c] for c in NTT_CLASSES)
    cf, F = ctx.ks_coarse_from, ctx.ks_fine_depth
    # per-prime digits need no recombination products (one conditional subtraction)
    per_unit = sum(0 if d <= F else DIGIT_PRODUCTS_PER_HMULT[8 if cf and d >= cf else ctx.ks_digit_primes]
                   for d in product_depths(wl["op"]))
    digit_products = per_unit * N * n_ct * wl.get("n_const", 1)
    ks_macs = works.get(8, 0.0)
    t_ideal = (butterflies + digit_products) / (mul_rate / MUL_PER_BUTTERFLY) + ks_macs / (mul_rate / MUL_PER_MAC)
    roof["path_frac"] = t_ideal / (ms_per_step / 1e3)
    roof["path_work_per_step"] = {"butterflies": butterflies, "digit_products": digit_products, "ks_macs": ks_macs,
                                  "ideal_ms": t_ideal * 1e3}
    # the same ideal against the part of the step outside the two tensor-core
    # conversion kernels, whose work the ideal leaves out
    tc = sum(shares.get(hp.PROFILE_CLASSES.index(c), 0.0) for c in ("lift", "scale_round")) / tot if tot else 0.0
    roof["tc_conversion_share"] = tc
    roof["path_frac_outside_tc"] = t_ideal / (ms_per_step / 1e3 * (1.0 - tc)) if tc < 1.0 else None
    # and with the conversions' MMA work at the measured dense bf16 (= f16) burst
    # peak: per coefficient 2 x 128 x 128 flops per MMA (M = 128 coefficients,
    # N = K = 128), two MMAs in the scale-and-round, one in the lift
    tc_flops = TC_FLOPS_PER_COEFF * (2 * works.get(hp.PROFILE_CLASSES.index("scale_round"), 0.0)
                                     + works.get(hp.PROFILE_CLASSES.index("lift"), 0.0))
    tflops = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] * 1e12
    roof["path_work_per_step"]["tc_flops"] = tc_flops
    roof["path_frac_with_tc"] = (t_ideal + tc_flops / tflops) / (ms_per_step / 1e3)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n_ct_per_gpu": n_ct, "slots_per_gpu": n_ct * N,
                       "tile_ct": ctx_tile(ctx), "ks_digit_primes": ctx.ks_digit_primes,
                       "ks_coarse_from": ctx.ks_coarse_from, "ks_fine_depth": ctx.ks_fine_depth,
                       "l2": "inputs larger than L2 (%.1f GB of ciphertexts read per step)"
                       % (n_ct * 2 * 15 * N * 8 * (2 if cy is not None else 1) / 1e9),
                       "parallelism": "replicas" if world == 1 else "dp%d (independent ciphertexts)" % world},
            "roofline": roof, "clocks": clk, "gpu_launches": launches,
            "kernel_shares": {hp.PROFILE_CLASSES[c]: shares[c] / tot for c in shares} if tot else None,
            "hmult_per_s": value / N * HMULT_PER_CT[wl["op"]]}

    # ---- end to end through the public API with pinned host buffers ----
    if not args.no_e2e and wl["op"] not in ("lt", "between", "in", "sum", "rotsum", "join"):
        line["e2e"] = e2e_measure(ctx, cx, cy, const_val, n_ct, N, args, world, dist)
    # ---- the headline line also carries config 3 (batched vs plain) and extras ----
    if wl["op"] == "ctct" and world == 1 and not (args.no_batched and args.no_extras) and not args.n_ct:
        del cx, cy, out
        torch.cuda.empty_cache()
        if not args.no_batched:
            r = batched_measure(ctx, 1, 1, stream)
            r["plain_elements_per_s"] = value
            r["packed_batched_over_plain"] = r["packed_batched_elements_per_s"] / value
            line["batched_vs_plain"] = r
        if not args.no_extras:
            line["extras"] = extras_measure(ctx, stream)
    # ---- CPU baseline (rank 0, N = 1 only) ----
    if not args.no_cpu and rank == 0 and world == 1:
        v, secs, desc = OracleSample(wl["op"], ctx.ks_digit_primes, ctx.ks_coarse_from, ctx.ks_fine_depth).time(4)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                                "cpu_seconds": secs}
        try:
            mc = multicore_baseline(wl["op"], dp=ctx.ks_digit_primes, cf=ctx.ks_coarse_from, F=ctx.ks_fine_depth)
            mc["speedup_over_one_core_sample"] = mc["value"] / v
        except Exception as e:  # the single-core baseline above stands on its own
            mc = {"value": None, "error": str(e)[:200]}
        line["cpu_baseline_multicore"] = mc
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def ctx_tile(ctx):
    return ctx.tile()


def extras_measure(ctx, stream):
    """More workloads at N = 32768, one timed pass each after one warm-up pass,
    each result checked against its closed form: config 4 (EQ against a constant
    over 2^28 slots = 8192 ciphertexts, three of them checked), and reduced
    sizes of every other row -- LT (Eq. 4) over 16 ciphertext pairs and BETWEEN
    over 8 ciphertexts with LT's key switching, IN (Eq. 6) against 8 constants
    over 32 ciphertexts, SUM WHERE over 128 ciphertext pairs, the rotate-and-add
    reduction of 64 ciphertexts and a JOIN of 8 A ciphertexts with 16 B rows
    and 2 attributes on the handle itself (every slot checked)."""
    import numpy as np
    import torch

    from paper_2602_24271_b300 import hp
    from paper_2602_24271_b300.inputs import eq_pair_columns

    N = ctx.N
    out = {}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # config 4: 2^28 slots against a constant (x drawn per chunk of 128 ciphertexts)
    n28, cval = 8192, 4242
    x28 = ctx.ct_empty(n28)
    probe = {}
    for c0 in range(0, n28, 128):
        xs, _ = eq_pair_columns(128 * N, seed=SEED_DATA + 1000 + c0)
        xs[::7] = cval
        x28[c0:c0 + 128] = ctx.encrypt(xs.reshape(128, N), seed=SEED_DATA + 3, ct_index0=c0)
        for c in (0, n28 // 2, n28 - 1):
            if c0 <= c < c0 + 128:
                probe[c] = xs[(c - c0) * N:(c - c0 + 1) * N]
    o28 = ctx.ct_empty(n28)
    ms = timed(lambda: ctx.run(hp.HP_EQ_CT_CONST, x28, None, cval, out=o28, stream=stream))
    dec = ctx.decrypt(o28[list(probe)])
    for k, c in enumerate(probe):
        assert np.array_equal(dec[k], (probe[c] == cval).astype(np.uint32)), "const28 result wrong"
    out["const28"] = {"workload": "EQ(x, c): 2^28 slots = 8192 ciphertexts vs a broadcast constant, N=32768",
                      "value": n28 * N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": 1, "warmup": 1,
                      "check": "closed form on ciphertexts 0, 4096, 8191"}
    del x28, o28
    torch.cuda.empty_cache()
    # LT over 16 ciphertext pairs, closed form on every slot, with LT's own key
    # switching (per-prime digits up to depth 4, five-prime digits, the two-digit
    # key from depth 10)
    lctx = ctx
    if (ctx.ks_fine_depth, ctx.ks_digit_primes, ctx.ks_coarse_from) != DEFAULT_KEY_SWITCHING["lt"]:
        F, dp, cf = DEFAULT_KEY_SWITCHING["lt"]
        lctx = hp.Context(LOGN, max_tile_ct=ctx_tile(ctx), ks_digit_primes=dp, ks_coarse_from=cf, ks_fine_depth=F)
        lctx.keygen(SEED_KEY)
    nl = 16
    xl, yl = eq_pair_columns(nl * N, seed=SEED_DATA + 7, value_bits=15)
    cxl = lctx.encrypt(xl.reshape(nl, N), seed=SEED_DATA + 4, ct_index0=0)
    cyl = lctx.encrypt(yl.reshape(nl, N), seed=SEED_DATA + 4, ct_index0=nl)
    ol = lctx.ct_empty(nl)
    ms = timed(lambda: lctx.run(hp.HP_LT, cxl, cyl, 0, out=ol, stream=stream))
    assert np.array_equal(lctx.decrypt(ol).reshape(-1), (xl < yl).astype(np.uint32)), "LT result wrong"
    out["lt"] = {"workload": "LT(x, y) (Eq. 4): 16 ciphertext pairs = 2^19 slots, x, y in [0, 2^15], N=32768, "
                 "511 multiplications per ciphertext (depth 18)", "value": nl * N / (ms / 1e3), "unit": UNIT,
                 "ms_per_step": ms, "steps": 1, "warmup": 1, "check": "closed form [x < y] on every slot",
                 "hmult_per_s": nl * 511 / (ms / 1e3), "ks_fine_depth": lctx.ks_fine_depth,
                 "ks_digit_primes": lctx.ks_digit_primes, "ks_coarse_from": lctx.ks_coarse_from}
    del cxl, cyl, ol
    # BETWEEN over 8 ciphertexts: two LT evaluations and their product
    nb, lo, hi = 8, 1000, 20000
    xb, _ = eq_pair_columns(nb * N, seed=SEED_DATA + 8, value_bits=15)
    cxb = lctx.encrypt(xb.reshape(nb, N), seed=SEED_DATA + 6, ct_index0=0)
    ob = lctx.ct_empty(nb)
    ms = timed(lambda: lctx.between(cxb, lo, hi, out=ob, stream=stream))
    assert np.array_equal(lctx.decrypt(ob).reshape(-1), ((xb >= lo) & (xb <= hi)).astype(np.uint32)), \
        "BETWEEN result wrong"
    out["between"] = {"workload": "x BETWEEN 1000 AND 20000: 8 ciphertexts = 2^18 slots, x in [0, 2^15], N=32768, "
                      "two LT evaluations and their product (1023 multiplications) per ciphertext",
                      "value": nb * N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": 1, "warmup": 1,
                      "check": "closed form [lo <= x <= hi] on every slot"}
    del cxb, ob
    if lctx is not ctx:
        lctx.close()
    torch.cuda.empty_cache()

    # the rows on the handle's own key switching
    ctx.galois_keygen(SEED_KEY)
    # IN against 8 constants drawn from the column, 32 ciphertexts
    ni, nk = 32, 8
    xi, _ = eq_pair_columns(ni * N, seed=SEED_DATA + 9)
    consts = [int(v) for v in xi[:nk]]
    cxi = ctx.encrypt(xi.reshape(ni, N), seed=SEED_DATA + 10, ct_index0=0)
    oi = ctx.ct_empty(ni)
    ms = timed(lambda: ctx.eq_fanout(cxi, consts, masks=False, in_set=oi, stream=stream))
    assert np.array_equal(ctx.decrypt(oi).reshape(-1), np.isin(xi, consts).astype(np.uint32)), "IN result wrong"
    out["in"] = {"workload": "IN(x, S) (Eq. 6), |S| = 8: 32 ciphertexts = 2^20 slots, 256 EQ chains, N=32768",
                 "value": ni * N * nk / (ms / 1e3), "unit": "slot-constant comparisons/s", "ms_per_step": ms,
                 "steps": 1, "warmup": 1, "check": "closed form [x in S] on every slot"}
    del cxi, oi
    # SUM(y) WHERE x = c over 128 ciphertext pairs: SELECT, then one rotate-and-add over the column
    ns, cval = 128, 4242
    xs, ys = eq_pair_columns(ns * N, seed=SEED_DATA + 11)
    xs[np.random.default_rng(SEED_DATA + 12).random(ns * N) < 0.25] = cval
    cxs = ctx.encrypt(xs.reshape(ns, N), seed=SEED_DATA + 13, ct_index0=0)
    cys = ctx.encrypt(ys.reshape(ns, N), seed=SEED_DATA + 13, ct_index0=ns)
    sel, agg = ctx.ct_empty(ns), ctx.ct_empty(1)

    def f_sum():
        ctx.run(hp.HP_SELECT, cxs, cys, cval, out=sel, stream=stream)
        ctx.rotate_sum(sel, group=ns, out=agg, stream=stream)

    ms = timed(f_sum)
    total = int(ys[xs == cval].astype(np.int64).sum() % 65537)
    assert np.all(ctx.decrypt(agg) == total), "SUM result wrong"
    out["sum"] = {"workload": "SUM(y) WHERE x = c: SELECT (Eq. 5) over 128 ciphertext pairs = 2^22 slots, then the "
                  "rotate-and-add reduction of the column into one ciphertext, N=32768",
                  "value": ns * N / (ms / 1e3), "unit": "slots/s", "ms_per_step": ms, "steps": 1, "warmup": 1,
                  "check": "the column's total in every slot"}
    # the rotate-and-add reduction of each of 64 ciphertexts (the SUM's y column)
    nr = 64
    orr = ctx.ct_empty(nr)
    ms = timed(lambda: ctx.rotate_sum(cys[:nr], out=orr, stream=stream))
    ref = ys[:nr * N].reshape(nr, N).astype(np.int64).sum(axis=1) % 65537
    assert np.array_equal(ctx.decrypt(orr), np.repeat(ref[:, None], N, axis=1).astype(np.uint32)), \
        "rotate-and-add result wrong"
    out["rotsum"] = {"workload": "rotate-and-add reduction (COUNT/SUM) of each of 64 ciphertexts = 2^21 slots, "
                     "15 rotations with key switching per ciphertext, N=32768",
                     "value": nr * N / (ms / 1e3), "unit": "slots reduced/s", "ms_per_step": ms, "steps": 1,
                     "warmup": 1, "check": "each ciphertext's total in every slot"}
    del cxs, cys, sel, agg, orr
    # JOIN: 8 A ciphertexts against 16 B rows with distinct keys from A's column, 2 attributes
    na, jr = 8, 16
    xa, _ = eq_pair_columns(na * N, seed=SEED_DATA + 14)
    bkey = np.zeros(N, dtype=np.uint32)
    bkey[:jr] = np.unique(xa[:64 * jr])[:jr]
    battr = np.random.default_rng(SEED_DATA + 15).integers(0, 65537, (2, N)).astype(np.uint32)
    cxa = ctx.encrypt(xa.reshape(na, N), seed=SEED_DATA + 16, ct_index0=0)
    cbk = ctx.encrypt(bkey.reshape(1, N), seed=SEED_DATA + 17, ct_index0=0)
    cba = [ctx.encrypt(battr[k].reshape(1, N), seed=SEED_DATA + 17, ct_index0=1 + k) for k in range(2)]
    jout = torch.empty((2, na, 2, 15, N), dtype=torch.int64, device="cuda")
    ms = timed(lambda: ctx.join(cxa, cbk, cba, jr, out=jout, stream=stream))
    for k in range(2):
        ref = np.zeros(na * N, dtype=np.uint32)
        for r in range(jr):
            ref[xa == bkey[r]] = battr[k][r]
        assert np.array_equal(ctx.decrypt(jout[k]).reshape(-1), ref), "JOIN result wrong"
    out["join"] = {"workload": "equi-join A.key = B.key (Extract + Broadcast): 8 A ciphertexts = 2^18 rows, 16 B "
                   "rows with 2 attributes (128 EQ chains, 256 products, 48 broadcasts), N=32768",
                   "value": na * N * jr / (ms / 1e3), "unit": "A-row x B-row comparisons/s", "ms_per_step": ms,
                   "steps": 1, "warmup": 1, "check": "both joined attribute columns on every slot"}
    del cxa, cbk, cba, jout
    torch.cuda.empty_cache()
    return out


def e2e_measure(ctx, cx, cy, const_val, n_ct, N, args, world, dist):
    import torch

    from paper_2602_24271_b300 import hp

    try:
        hx = torch.empty(cx.shape, dtype=torch.int64, pin_memory=True)
        hx.copy_(cx)
        hy = None
        if cy is not None:
            hy = torch.empty(cy.shape, dtype=torch.int64, pin_memory=True)
            hy.copy_(cy)
        ho = torch.empty(cx.shape, dtype=torch.int64, pin_memory=True)
    except RuntimeError as e:
        return {"value": None, "unit": UNIT, "error": "pinned host allocation failed: %s" % str(e)[:120]}
    op = hp.HP_EQ_CT_CT if cy is not None else hp.HP_EQ_CT_CONST
    ctx.run(op, hx[:1], hy[:1] if hy is not None else None, const_val, out=ho[:1])  # warm the host path
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.run(op, hx, hy, const_val, out=ho)
    secs = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, device="cuda")
    word = 8
    h2d = n_ct * 2 * 15 * N * word * (2 if cy is not None else 1)
    d2h = n_ct * 2 * 15 * N * word
    return {"value": n_ct * N * world / secs, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "seconds_per_step": secs, "path": "hp_run with pinned host buffers (library stages tiles through HBM)"}


def batched_measure(ctx, steps: int, warm: int, stream, per_instance: bool = True):
    """Config 3: 4096 uneven instances (sizes log-uniform in [2^8, 2^16] slots,
    dictionary IDs) through hp_run_batched, slot-packed into shared ciphertexts
    and (per_instance) with one group of ciphertexts per instance, against plain
    hp_run calls per instance.  elements = slots of the instances (the rows
    compared).  Checks the closed form on sampled instances of each form."""
    import numpy as np
    import torch

    from paper_2602_24271_b300 import hp
    from paper_2602_24271_b300.inputs import dictionary_column, log_uniform_sizes

    N = ctx.N
    sizes = log_uniform_sizes(4096, seed=2, lo_log2=8, hi_log2=16)
    total = int(sizes.sum())
    rng = np.random.default_rng(2)

    def columns(n):
        x = dictionary_column(n, seed=2)
        other = dictionary_column(n, seed=3)
        y = np.where(rng.random(n) < 0.5, x, other).astype(np.uint32)
        return x, y

    def encrypt_all(slots, n_ct, idx0):
        out = ctx.ct_empty(n_ct)
        for c0 in range(0, n_ct, 128):
            c1 = min(n_ct, c0 + 128)
            out[c0:c1] = ctx.encrypt(slots[c0 * N:c1 * N].reshape(-1, N), seed=SEED_DATA, ct_index0=idx0 + c0)
        return out

    def timed(fn, n_steps, n_warm):
        for _ in range(n_warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n_steps

    launches = {}
    # (a) slot-packed: instances back to back in one global slot space
    packed, off = [], 0
    for n in sizes:
        ct0, so = off // N, off % N
        packed.append((ct0, (so + int(n) + N - 1) // N, so, int(n), 0, 0))
        off += int(n)
    n_pk = (off + N - 1) // N
    xs, ys = columns(n_pk * N)
    px, py = encrypt_all(xs, n_pk, 0), encrypt_all(ys, n_pk, n_pk)
    pout = ctx.ct_empty(n_pk)

    def f_packed():
        ctx.run_batched(hp.HP_EQ_CT_CT, packed, px, py, out=pout, stream=stream)
        launches["packed"] = ctx.launch_count()

    ms_packed = timed(f_packed, steps, warm)
    dec_p = ctx.decrypt(pout[:4]).reshape(-1)
    for (ct0, k, so, n, _, _) in packed[:8]:
        g0 = ct0 * N + so
        if g0 + n <= 4 * N:
            assert np.array_equal(dec_p[g0:g0 + n], (xs[g0:g0 + n] == ys[g0:g0 + n]).astype(np.uint32))
    res = {"instances": 4096, "instance_slots": total, "ciphertexts_packed": n_pk,
           "packed_batched_elements_per_s": total / (ms_packed / 1e3), "packed_ms_per_pass": ms_packed}
    del px, py, pout
    if per_instance:
        # (b) one group of ciphertexts per instance; (c) plain hp_run per instance
        per, c = [], 0
        for n in sizes:
            k = (int(n) + N - 1) // N
            per.append((c, k, 0, int(n), 0, 0))
            c += k
        n_pi = c
        xi, yi = columns(n_pi * N)
        ix, iy = encrypt_all(xi, n_pi, 0), encrypt_all(yi, n_pi, n_pi)
        iout = ctx.ct_empty(n_pi)

        def f_per():
            ctx.run_batched(hp.HP_EQ_CT_CT, per, ix, iy, out=iout, stream=stream)
            launches["per"] = ctx.launch_count()

        def f_plain():
            n = 0
            for (c0, k, _, _, _, _) in per:
                ctx.run(hp.HP_EQ_CT_CT, ix[c0:c0 + k], iy[c0:c0 + k], 0, out=iout[c0:c0 + k], stream=stream)
                n += ctx.launch_count()
            launches["plain"] = n

        ms_per = timed(f_per, 1, 1)
        ms_plain = timed(f_plain, 1, 0)
        dec_i = ctx.decrypt(iout[:2]).reshape(-1)
        assert np.array_equal(dec_i[:N], (xi[:N] == yi[:N]).astype(np.uint32))
        res.update({"ciphertexts_per_instance": n_pi,
                    "per_instance_batched_elements_per_s": total / (ms_per / 1e3),
                    "plain_per_instance_calls_elements_per_s": total / (ms_plain / 1e3),
                    "packed_over_plain_per_instance_calls": ms_plain / ms_packed,
                    "per_instance_batched_over_plain_per_instance_calls": ms_plain / ms_per})
        del ix, iy, iout
    res["error"] = "bit-exact (integer arithmetic; parity tests vs the oracle)"
    res["launches_by_form"] = dict(launches)
    torch.cuda.empty_cache()
    return res


def run_batched(args):
    """Config 3 on its own line: the packed batched form is the value."""
    import torch

    from paper_2602_24271_b300 import hp

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wl = workload("batched")
    ctx = hp.Context(LOGN, max_tile_ct=args.tile, ks_digit_primes=digit_primes(args, "batched"),
                     ks_coarse_from=coarse_from(args, "batched"), ks_fine_depth=fine_depth(args, "batched"))
    ctx.keygen(SEED_KEY)
    tile = ctx.autotune()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    r = batched_measure(ctx, args.steps, args.warmup, stream)
    clk = clocks.stop()
    ctx.check_status()
    value = r["packed_batched_elements_per_s"]
    cpu = None
    if not args.no_cpu:
        v, secs, desc = OracleSample("batched", ctx.ks_digit_primes, ctx.ks_coarse_from, ctx.ks_fine_depth).time(4)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, "cpu_seconds": secs}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["packed_ms_per_pass"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl["desc"], "instances": r["instances"], "instance_slots": r["instance_slots"],
                       "ciphertexts_packed": r["ciphertexts_packed"],
                       "ciphertexts_per_instance": r["ciphertexts_per_instance"], "tile_ct": tile,
                       "l2": "inputs larger than L2"},
            "batched_vs_plain": r, "clocks": clk,
            "gpu_launches": r["launches_by_form"].get("packed", 0) * args.steps,
            "hmult_per_s": r["ciphertexts_packed"] * 16 / (r["packed_ms_per_pass"] / 1e3)}
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batched":
        run_batched(args)
    else:
        run_libhp(args)


if __name__ == "__main__":
    main()
