"""The benchmark's reference arm runs on the CPU alone: `bench.py --impl
reference` times the oracle on every host core (spawned processes updating
disjoint site subsets of each half-sweep) and prints one JSON line with the
contract's keys.  Also checks that the multi-process half-sweep equals the
oracle's own single-process half-sweep bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3"], capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["cpu_model"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_pooled_half_sweep_equals_oracle():
    sys.path.insert(0, ROOT)
    import bench
    L = (4, 4, 6, 4)
    oracle.build()
    U0 = oracle.hot_start(L, 3)
    ref = U0.copy()
    oracle.half_sweep(L, 5.7, 9, 2, 1, 1, ref)
    pool = bench.OraclePool(L, U0, procs=3)
    try:
        n = pool.half_sweep(5.7, 9, 2, 1, 1)
        got = np.array(pool.U)
    finally:
        pool.close()
    assert n == int(np.prod(L)) // 2
    assert np.array_equal(got, ref)
