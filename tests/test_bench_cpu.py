"""Host-side pieces of bench.py (CPU only): the workload table, the stored
ncu traffic lookup and the reference arm's JSON line, which times the oracle
on a bounded sample and needs no GPU."""
import json
import os
import subprocess
import sys

import pytest

import bench

OPS = ["ctct", "const", "batched", "in", "lt", "between", "sum", "rotsum", "join"]
CONFIGS = ["plain", "const28", "batched", "lt", "between", "in", "sum", "rotsum", "join"]


def test_every_config_has_a_composition_and_a_multiplication_count():
    ops = {bench.workload(c)["op"] for c in CONFIGS}
    assert ops == set(OPS)
    for op in OPS:
        assert op in bench.OracleSample.COUNTS
        assert op == "batched" or op in bench.HMULT_PER_CT
    for op in OPS:  # the multiplications' depths agree with the counts
        assert op == "batched" or len(bench.product_depths(op)) == bench.HMULT_PER_CT[op]
    # an EQ chain is 16 squarings (p - 1 = 2^16, Eq. 3), at depths 1 .. 16
    assert bench.product_depths("ctct") == list(range(1, 17)) and bench.HMULT_PER_CT["ctct"] == 16
    # LT's schedule: 511 products, the deepest at 18; 255 of them at depth 10 or more
    d = bench.lt_product_depths()
    assert len(d) == 511 == bench.HMULT_PER_CT["lt"] and max(d) == 18 and sum(v >= 10 for v in d) == 255
    # BETWEEN: two LT evaluations and their product at depth 19 (Sec. 4.2.2)
    assert bench.HMULT_PER_CT["between"] == 2 * 511 + 1 and max(bench.product_depths("between")) == 19


def test_stored_traffic_scales_with_the_tile_and_follows_the_sources():
    path = os.path.join(bench.ROOT, "profiles", "ncu_counters.json")
    d = json.load(open(path))
    tile = d["tile_ct"]
    for kernel, k in d["kernels"].items():
        want = k["dram_bytes_per_launch_full"]
        got = bench.load_traffic(kernel, tile)
        if k["source_hash"] == bench.source_hash(kernel):
            assert got == pytest.approx(want)
            assert bench.load_traffic(kernel, 2 * tile) == pytest.approx(2 * want)
        else:
            assert got is None  # counters taken on other kernel sources are not reported
    assert bench.load_traffic("k_no_such_kernel", tile) is None


@pytest.mark.parametrize("config", ["plain", "rotsum"])  # multiplications; rotations with a Galois key
def test_reference_arm_prints_one_json_line(config):
    env = dict(os.environ, RANK="0")
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--config", config,
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["config"]["workload"] == bench.workload(config)["desc"]
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    env = dict(os.environ, RANK="1")
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""
