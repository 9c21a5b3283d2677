"""The ncu records bench.py reads (profiles/stencil_traffic.txt): every
record is one capture of one workload and decomposition, so that a record
appended without its blank separator cannot silently merge into the one
before it (the later keys would overwrite the earlier ones)."""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _records():
    path = os.path.join(ROOT, "profiles", "stencil_traffic.txt")
    recs, cur = [], []
    for line in open(path):
        if not line.strip():
            if cur:
                recs.append(cur)
            cur = []
        elif not line.startswith("#"):
            cur.append(line.rstrip("\n"))
    if cur:
        recs.append(cur)
    return recs


def test_each_record_is_one_capture():
    recs = _records()
    assert recs
    for rec in recs:
        keys = [ln.split(":", 1)[0].strip() for ln in rec if ":" in ln]
        assert len(keys) == len(set(keys)), rec[:3]
        assert "stencil_source_sha256_16" in keys and "points_per_thread" in keys and "capture" in keys
        assert "dram_bytes_per_update" in keys or "instructions_per_point_iteration" in keys


def test_lookup_keys_are_unique_per_source():
    seen = set()
    for rec in _records():
        d = dict(ln.split(":", 1) for ln in rec if ":" in ln)
        d = {k.strip(): v.strip() for k, v in d.items()}
        key = (d["stencil_source_sha256_16"], d.get("workload", "sphere-union"), d["points_per_thread"])
        assert key not in seen, key
        seen.add(key)
