"""Host-side helpers of bench.py (no GPU): the workload record, the ncu traffic lookup and the
schedule options carried in the JSON line's config."""
import argparse
import glob
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _args(**kw):
    a = argparse.Namespace(n=16384, levels=2, variant="split3", algo="auto", schedule="auto", round_tiles=0)
    for key, v in kw.items():
        setattr(a, key, v)
    return a


def test_config_names_the_workload_and_the_work_order():
    d = bench.config_dict(_args(), 16384)
    assert d["workload"] == "strassen-L2-split3-square-m16384-n16384-k16384"
    assert (d["m"], d["n"], d["k"], d["levels"]) == (16384, 16384, 16384, 2)
    assert d["schedule"] == "auto" and d["round_tiles"] == 0
    d = bench.config_dict(_args(schedule="product", round_tiles=152, levels=1), 2048)
    assert d["workload"] == "strassen-L1-split3-rank-k-m16384-n16384-k2048"
    assert d["schedule"] == "product" and d["round_tiles"] == 152


def test_recorded_traffic_follows_the_kernel_sources():
    """The traffic record is reported only while the hashed kernel sources are unchanged; an
    unknown workload has none."""
    assert bench.recorded_traffic("no-such-workload") is None
    recs = glob.glob(os.path.join(ROOT, "profiles", "*_traffic_*.json"))
    assert recs
    for path in recs:
        with open(path) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["source_files"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        got = bench.recorded_traffic(rec["workload"])
        if h.hexdigest() == rec["source_sha256"]:
            assert got == rec["dram_bytes_read"] + rec["dram_bytes_write"]
        else:
            assert got is None
