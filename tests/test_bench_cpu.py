"""The benchmark's reference arm (the FP64 oracle on the host cores) and its
JSON line, on CPU: the fields every bench line carries, and the non-zero
ranks of a multi-rank launch leaving without work or output."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                           "--workload", "tiny"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "slr_subdomain_bounds_per_sec" and line["unit"] == "boxes/s"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["steps"] == 1 and line["warmup"] == 0 and line["n_gpus"] == 1
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert line["config"]["workload"].startswith("tiny_2-8-8-1 D=16")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_parity_field_compares_levels_and_bracket():
    """bench.parity_of: equal when every level the oracle finished and the
    bracket agree; a differing level or bracket is reported (CPU)."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from workloads import generators as gen
    p = gen.tiny(0)
    D = 10
    want = oracle.count(p.net, p.lo, p.hi, p.prop, D)
    ref = {"levels": want.levels, "complete": True, "unsafe_lo": want.unsafe_lo, "unsafe_hi": want.unsafe_hi}
    gpu = {"unsafe_lo": want.unsafe_lo, "unsafe_hi": want.unsafe_hi}
    for k in ("boxes", "safe", "unsafe", "undecided"):
        gpu["level_" + k] = [lv[k] for lv in want.levels]
    assert bench.parity_of(gpu, ref, D)["equal"]
    bad = dict(gpu, level_safe=list(gpu["level_safe"]))
    bad["level_safe"][5] += 1
    r = bench.parity_of(bad, ref, D)
    assert not r["equal"] and r["first_differing_level"] == 5
    r = bench.parity_of(dict(gpu, unsafe_hi=gpu["unsafe_hi"] + 1), ref, D)
    assert not r["equal"] and r["levels_equal"] and not r["bracket_equal"]
    part = dict(ref, levels=want.levels[:4], complete=False)
    r = bench.parity_of(gpu, part, D)
    assert r["equal"] and r["levels_compared"] == 4 and "oracle_lo" not in r
