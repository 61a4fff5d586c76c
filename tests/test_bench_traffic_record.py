"""bench.py's recorded DRAM traffic (the roofline's `traffic`) is tied to the code it was
captured on: a hash of the kernel sources without their comments.  Editing a comment keeps the
record; editing code drops it (the line then reports null)."""
import json

import bench


SRC = "int f(int x) {  // twice\n    return 2 * x;  /* doubled */\n}\n"


def test_code_hash_ignores_comments_and_layout():
    a = bench._code_only(SRC)
    assert a == bench._code_only(SRC.replace("// twice", "// times two").replace("doubled", "x2"))
    assert a == bench._code_only(SRC.replace("    return", "  return"))
    assert a != bench._code_only(SRC.replace("2 * x", "3 * x"))


def test_recorded_traffic_follows_the_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1708_07853_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    files = bench.KERNEL_SOURCES["fwd_l1_cdf97_f32"]
    for k, f in enumerate(files):
        (csrc / f).write_text(SRC.replace("2 * x", f"{k + 2} * x"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.src_hash("fwd_l1_cdf97_f32")
    rec = {"fwd_l1_cdf97_f32": {"src_hash": h, "dram_bytes_per_launch": 123}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("fwd_l1_cdf97_f32") == 123
    (csrc / files[0]).write_text(SRC.replace("// twice", "// a new comment").replace("2 * x", "2 * x"))
    assert bench.recorded_traffic("fwd_l1_cdf97_f32") == 123  # comment only
    (csrc / files[0]).write_text(SRC.replace("2 * x", "7 * x"))
    assert bench.recorded_traffic("fwd_l1_cdf97_f32") is None  # code changed

