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
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ncu-region", action="store_true",
                    help="after warm-up, run one extra step between cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


def workload(cfg: str):
    if cfg == "between":
        return dict(n_ct=64, op="between", desc="x BETWEEN 1000 AND 20000 (Sec. 4.2.2: 1 - LT(x, lo) - LT(hi, x)): "
                    "2^21 slots = 64 BFV ciphertexts, x in [0, 2^15], N=32768, L=15, p=65537; two LT evaluations "
                    "(1022 multiplications) per ciphertext, bit-exact")
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
HMULT_PER_CT = {"ctct": 16, "const": 16, "in": 16, "lt": 511, "between": 1022, "sum": 17, "rotsum": 0, "join": 18}


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
class OracleSample:
    """One ciphertext of the workload (N = 32768) on the CPU oracle, keys and
    encryptions made once.  `time(n_mul)` times the oracle's primitives on it
    single-threaded (difference, `n_mul` multiplications with relinearisation,
    "1 -", and one rotation with key switching where the workload rotates) and
    composes the time of one unit of the workload from the counts below.  The
    composition counts the multiplications and rotations the workload performs
    and the difference and "1 -" of each EQ chain; ciphertext additions, the
    plaintext products of Extract and LT's inner sums (255 scalar products per
    giant step) are left out, so for those workloads the rate is an upper bound
    on the oracle's."""

    # per ciphertext (per ciphertext and B row for join): (differences, multiplications,
    # "1 -", rotations, what is left out)
    COUNTS = {
        "ctct": (1, 16, 1, 0, ""),
        "const": (1, 16, 1, 0, ""),
        "batched": (1, 16, 1, 0, ""),
        "in": (1, 16, 1, 0, "the additions of the IN sum"),
        "lt": (1, 511, 0, 0, "the 128 inner sums of 255 scalar products and the additions"),
        "between": (3, 1022, 1, 0, "the 2 x 128 inner sums of 255 scalar products and the additions"),
        "sum": (1, 17, 1, 15 / 2048, "the additions"),
        "rotsum": (0, 0, 0, 15, "the additions"),
        "join": (1, 18, 1, 45 / 64, "the plaintext products of Extract and the additions"),
    }

    def __init__(self, op: str = "ctct"):
        import oracle
        from paper_2602_24271_b300.inputs import eq_pair_columns

        self.op = op
        self.o = oracle.Oracle(LOGN)
        self.o.keygen(SEED_KEY)
        x, y = eq_pair_columns(self.o.N, seed=SEED_DATA)
        self.cx, self.cy = self.o.encrypt(x, 7, 0), self.o.encrypt(y, 7, 1)
        self.g = None
        if self.COUNTS[op][3]:
            self.g = self.o.galois_elements()[0]
            self.o.galois_keygen(SEED_KEY, self.g)

    def time(self, n_mul: int = 1):
        o = self.o
        n_sub, n_m, n_1m, n_rot, left_out = self.COUNTS[self.op]
        n_mul = n_mul if n_m else 0  # a workload without multiplications times none
        t0 = time.perf_counter()
        d = o.sub(self.cx, self.cy)
        t1 = time.perf_counter()
        for _ in range(n_mul):
            d = o.mul_relin(d, d)
        t2 = time.perf_counter()
        o.one_minus(d)
        t3 = time.perf_counter()
        t_rot = 0.0
        if self.g is not None:
            o.rotate(d, self.g)
            t_rot = time.perf_counter() - t3
        t_sub, t_mul, t_1m = t1 - t0, (t2 - t1) / max(1, n_mul), t3 - t2
        per_unit = n_sub * t_sub + n_m * t_mul + n_1m * t_1m + n_rot * t_rot
        desc = ("1 ciphertext at N=32768 (32768 slots) on the oracle, single-threaded: a difference, %d "
                "multiplication(s) with relinearisation, '1 -'%s timed; one unit of the workload composed as "
                "%d difference(s) + %d multiplications + %d x '1 -'%s%s" % (
                    n_mul, " and one rotation" if self.g is not None else "", n_sub, n_m, n_1m,
                    " + %.3g rotations" % n_rot if n_rot else "",
                    "; not counted: %s (the rate is an upper bound)" % left_out if left_out else ""))
        return o.N / per_unit, time.perf_counter() - t0, desc


def _oracle_worker(op, n_mul, barrier, results):
    sample = OracleSample(op)
    barrier.wait(timeout=120)  # every worker set up: the timed samples run concurrently
    results.put(sample.time(n_mul))


def multicore_baseline(op: str, n_mul: int = 1, max_workers: int = 32):
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
    procs = [ctx.Process(target=_oracle_worker, args=(op, n_mul, barrier, results)) for _ in range(w)]
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
    sample = OracleSample(wl["op"])
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
    ctx = hp.Context(LOGN, max_tile_ct=args.tile)
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
    shares = {}
    for c, name in enumerate(hp.PROFILE_CLASSES):
        ms, n, w = ctx.profile_read(c)
        shares[c] = ms
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
    roof["traffic"] = load_traffic(kernel, ctx_tile(ctx))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n_ct_per_gpu": n_ct, "slots_per_gpu": n_ct * N,
                       "tile_ct": ctx_tile(ctx), "l2": "inputs larger than L2 (%.1f GB of ciphertexts read per step)"
                       % (n_ct * 2 * 15 * N * 8 * (2 if cy is not None else 1) / 1e9),
                       "parallelism": "replicas" if world == 1 else "dp%d (independent ciphertexts)" % world},
            "roofline": roof, "clocks": clk, "gpu_launches": launches,
            "kernel_shares": {hp.PROFILE_CLASSES[c]: shares[c] / tot for c in shares} if tot else None,
            "hmult_per_s": value / N * HMULT_PER_CT[wl["op"]]}

    # ---- end to end through the public API with pinned host buffers ----
    if not args.no_e2e and wl["op"] not in ("lt", "between", "in", "sum", "rotsum", "join"):
        line["e2e"] = e2e_measure(ctx, cx, cy, const_val, n_ct, N, args, world, dist)
    # ---- CPU baseline (rank 0, N = 1 only) ----
    if not args.no_cpu and rank == 0 and world == 1:
        v, secs, desc = OracleSample(wl["op"]).time(8)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                                "cpu_seconds": secs}
        try:
            mc = multicore_baseline(wl["op"])
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


def run_batched(args):
    """Config 3: uneven instances through hp_run_batched (slot-packed and one
    ciphertext group per instance) against plain hp_run calls per instance.
    elements = slots of the instances (the real rows compared)."""
    import numpy as np
    import torch

    from paper_2602_24271_b300 import hp
    from paper_2602_24271_b300.inputs import dictionary_column, log_uniform_sizes

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wl = workload("batched")
    ctx = hp.Context(LOGN, max_tile_ct=args.tile)
    ctx.keygen(SEED_KEY)
    tile = ctx.autotune()
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
    # (b) one group of ciphertexts per instance
    per, c = [], 0
    for n in sizes:
        k = (int(n) + N - 1) // N
        per.append((c, k, 0, int(n), 0, 0))
        c += k
    n_pi = c
    xi, yi = columns(n_pi * N)
    ix, iy = encrypt_all(xi, n_pi, 0), encrypt_all(yi, n_pi, n_pi)
    iout = ctx.ct_empty(n_pi)
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    launches = {}

    def f_packed():
        ctx.run_batched(hp.HP_EQ_CT_CT, packed, px, py, out=pout, stream=stream)
        launches["packed"] = ctx.launch_count()

    def f_per():
        ctx.run_batched(hp.HP_EQ_CT_CT, per, ix, iy, out=iout, stream=stream)
        launches["per"] = ctx.launch_count()

    def f_plain():
        n = 0
        for (c0, k, _, _, _, _) in per:
            ctx.run(hp.HP_EQ_CT_CT, ix[c0:c0 + k], iy[c0:c0 + k], 0, out=iout[c0:c0 + k], stream=stream)
            n += ctx.launch_count()
        launches["plain"] = n

    ms_packed = timed(f_packed, args.steps, args.warmup)
    ms_per = timed(f_per, 1, 1)
    ms_plain = timed(f_plain, 1, 0)
    clk = clocks.stop()
    ctx.check_status()
    # closed form on sampled instances of each form
    dec_p = ctx.decrypt(pout[:4]).reshape(-1)
    for (ct0, k, so, n, _, _) in packed[:8]:
        g0 = ct0 * N + so
        if g0 + n <= 4 * N:
            assert np.array_equal(dec_p[g0:g0 + n], (xs[g0:g0 + n] == ys[g0:g0 + n]).astype(np.uint32))
    dec_i = ctx.decrypt(iout[:2]).reshape(-1)
    assert np.array_equal(dec_i[:N], (xi[:N] == yi[:N]).astype(np.uint32))
    value = total / (ms_packed / 1e3)
    cpu = None
    if not args.no_cpu:
        v, secs, desc = OracleSample("batched").time(8)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, "cpu_seconds": secs}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_packed, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "instances": 4096, "instance_slots": total, "ciphertexts_packed": n_pk,
                       "ciphertexts_per_instance": n_pi, "tile_ct": tile, "l2": "inputs larger than L2"},
            "batched_vs_plain": {
                "packed_batched_elements_per_s": value,
                "per_instance_batched_elements_per_s": total / (ms_per / 1e3),
                "plain_per_instance_calls_elements_per_s": total / (ms_plain / 1e3),
                "packed_over_plain": ms_plain / ms_packed,
                "per_instance_batched_over_plain": ms_plain / ms_per,
                "error": "bit-exact (integer arithmetic; parity tests vs the oracle)"},
            "clocks": clk, "gpu_launches": launches.get("packed", 0) * args.steps,
            "gpu_launches_by_form": launches, "hmult_per_s": n_pk * 16 / (ms_packed / 1e3)}
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
