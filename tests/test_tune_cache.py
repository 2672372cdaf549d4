"""The autotuner's table on the CPU: the key's buckets, the JSON file round trip, and a second
process picking the entry up through DJ_TUNE_FILE.  No GPU: these calls only touch host state."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dj():
    from paper_2504_03667_gb300 import build, dj as _dj
    build.build()
    _dj.load_library()
    return _dj


def _file(path, entries):
    with open(path, "w") as f:
        json.dump({"version": 1, "entries": entries}, f)


def test_buckets_and_round_trip(dj, tmp_path):
    src = tmp_path / "tune.json"
    # n bucket floor(log2 n): 8192 -> 13; density bucket floor(log2(n^2 / entries)): 1/20 -> 4, 1/2 -> 1
    _file(src, [{"n_bucket": 13, "density_bucket": 4, "sms": 152, "engine": "lockstep", "cluster_size": 0,
                 "threads": 512, "ms": 3.5},
                {"n_bucket": 14, "density_bucket": 1, "sms": 152, "engine": "cluster", "cluster_size": 16,
                 "threads": 256, "ms": 40.0},
                {"n_bucket": 9, "density_bucket": 0, "sms": 148, "engine": "cluster", "cluster_size": 99}])  # bad size
    dj.dj_tune_load(str(src))
    n = 8192
    assert dj.dj_tune_lookup(n, int(0.05 * n * n), 152) == {"engine": "lockstep", "cluster_size": 0}
    assert dj.dj_tune_lookup(n + 5000, int(0.05 * (n + 5000) ** 2), 152)["engine"] == "lockstep"  # same buckets
    assert dj.dj_tune_lookup(n, int(0.05 * n * n), 148) is None  # another SM count
    assert dj.dj_tune_lookup(n, int(0.5 * n * n), 152) is None   # another density bucket
    assert dj.dj_tune_lookup(16384, int(0.5 * 16384 ** 2), 152) == {"engine": "cluster", "cluster_size": 16}
    assert dj.dj_tune_lookup(16383, int(0.5 * 16384 ** 2), 152) is None  # n bucket 13
    assert dj.dj_tune_lookup(600, 600 * 600, 148) is None  # the entry with an invalid cluster size was dropped
    out = tmp_path / "saved.json"
    dj.dj_tune_save(str(out))
    saved = json.loads(out.read_text())
    keys = {(e["n_bucket"], e["density_bucket"], e["sms"]): e for e in saved["entries"]}
    assert keys[(13, 4, 152)]["engine"] == "lockstep" and keys[(14, 1, 152)]["cluster_size"] == 16
    # a fresh process reads the saved file through the environment variable
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2504_03667_gb300 import dj\n"
            "print(dj.dj_tune_lookup(8192, int(0.05 * 8192 * 8192), 152))\n"
            "print(dj.dj_tune_lookup(16384, int(0.5 * 16384 ** 2), 152))\n" % ROOT)
    env = dict(os.environ, DJ_TUNE_FILE=str(out))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    assert lines[0] == "{'engine': 'lockstep', 'cluster_size': 0}"
    assert lines[1] == "{'engine': 'cluster', 'cluster_size': 16}"


def test_unreadable_file_is_an_error(dj, tmp_path):
    with pytest.raises(dj.DjError) as ei:
        dj.dj_tune_load(str(tmp_path / "missing.json"))
    assert ei.value.status == dj.DJ_EINVAL
