"""Tuning-table file handling (CPU only: no device calls)."""
import json

from paper_2010_02994_gb300 import tuning


def test_bucket_is_ceil_log2():
    assert tuning.bucket(1) == 0 and tuning.bucket(2) == 1 and tuning.bucket(1000) == 10
    assert tuning.bucket(1024) == 10 and tuning.bucket(1025) == 11 and tuning.bucket(100_000) == 17


def test_save_merges_entries(tmp_path, monkeypatch):
    monkeypatch.setattr(tuning, "gpu_name", lambda device=0: "TEST GPU")
    path = str(tmp_path / "t.json")
    tuning.save([{"d": 2, "bucket": 17, "warps": 8, "col_groups": 1, "ctas_per_sm": 0, "ms": 6.5}], path=path)
    tuning.save([{"d": 2, "bucket": 17, "warps": 4, "col_groups": 2, "ctas_per_sm": 2, "ms": 6.0},
                 {"d": 4, "bucket": 14, "warps": 4, "col_groups": 1, "ctas_per_sm": 0, "ms": 1.0}], path=path)
    table = json.load(open(path))
    assert [(e["d"], e["bucket"], e["warps"]) for e in table["TEST GPU"]] == [(2, 17, 4), (4, 14, 4)]
    assert tuning.read(str(tmp_path / "missing.json")) == {}
