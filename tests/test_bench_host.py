"""Host logic of bench.py that needs no GPU: the launch-mode labels read from a
plan's launch shape, and the ncu traffic records, which count only while the
kernel sources they name hash to the recorded value."""
import hashlib
import os
import shutil

import bench


def test_launch_labels():
    assert bench._launch_label(-2) == "split"
    assert bench._launch_label(-1) == "resident"
    assert bench._launch_label(0) == "persistent"
    assert bench._launch_label(4) == "graph"
    assert bench._launch_label(16 + 3) == "graph+pdl"


def _copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2502_12878_gb300", "csrc")
    dst = tmp_path / "paper_2502_12878_gb300" / "csrc"
    dst.mkdir(parents=True)
    for name in ("step.cuh", "step_res.cuh", "step_split.cuh"):
        shutil.copy(os.path.join(src, name), dst / name)
    (tmp_path / "profiles").mkdir()
    return dst


def _record(tmp_path, sources, sha, value=123456789):
    lines = ["# a traffic record", f"traffic_bytes_per_launch = {value}"]
    if sources is not None:
        lines.append("kernel_sources = " + ",".join(sources))
    lines.append(f"kernel_source_sha1 = {sha}")
    (tmp_path / "profiles" / "rec.txt").write_text("\n".join(lines) + "\n")


def test_traffic_record_counts_only_for_its_sources(tmp_path, monkeypatch):
    csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    names = ["step.cuh", "step_res.cuh", "step_split.cuh"]
    h = hashlib.sha1()
    for n in names:
        h.update((csrc / n).read_bytes())
    _record(tmp_path, names, h.hexdigest())
    assert bench._traffic("rec.txt") == 123456789
    # the same files in another order, or one file changed: the record no longer counts
    _record(tmp_path, names[::-1], h.hexdigest())
    assert bench._traffic("rec.txt") is None
    _record(tmp_path, names, h.hexdigest())
    (csrc / "step_split.cuh").write_bytes((csrc / "step_split.cuh").read_bytes() + b"\n")
    assert bench._traffic("rec.txt") is None
    # a record without a source list hashes step.cuh alone
    _record(tmp_path, None, hashlib.sha1((csrc / "step.cuh").read_bytes()).hexdigest(), 42)
    assert bench._traffic("rec.txt") == 42
    assert bench._traffic("missing.txt") is None


def test_committed_split_record_is_well_formed():
    rec = {}
    for line in open(os.path.join(bench.ROOT, "profiles", "split64_traffic.txt")):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            rec[k.strip()] = v.strip()
    assert int(rec["traffic_bytes_per_launch"]) > 0
    assert rec["kernel_sources"].split(",") == ["step.cuh", "step_res.cuh", "step_split.cuh"]
    assert len(rec["kernel_source_sha1"]) == 40
