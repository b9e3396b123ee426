"""bench.py's reference arm (the oracle timed on host cores) prints one JSON line with
the keys of the benchmark contract, on CPU, for a small workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"metric", "value", "unit", "impl", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline",
        "e2e"}


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "small", "--steps", "2", "--warmup", "1",
                          "--cpu-queries", "8"], cwd=ROOT, check=True, capture_output=True,
                         text=True, timeout=600).stdout.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    ac = cb["all_cores"]                  # the same oracle on every host core, when several
    assert ac is None or (ac["cores"] >= 2 and ac["value"] > 0 and ac["queries"] == 8 * ac["cores"])
    assert line["config"]["workload"] == "small-20k-d128"


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "small", "--steps", "1", "--warmup", "0"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_workload_label_names_the_actual_shape():
    # a run that overrides n or D reports its own shape, and the label of the default
    # GIST-like run is the key the recorded DRAM traffic is stored under
    sys.path.insert(0, ROOT)
    import bench
    import datagen
    assert bench.workload_label(datagen.workload("gist")) == "gist-like-1M-d960"
    assert bench.workload_label(datagen.workload("gist", n=6_000_000, D=160)) == "gist-like-6M-d160"
    assert bench.workload_label(datagen.workload("deep")) == "deep-like-10M-d96-zipf"
    assert bench.workload_label(datagen.workload("serve", n=200_000)) == "msmarco-like-200k-d1024"
    assert all(key[1] == "gist-like-1M-d960" for key in bench.NCU_TRAFFIC)
