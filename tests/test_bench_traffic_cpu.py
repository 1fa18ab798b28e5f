"""The bench's link between ncu summaries and the code (CPU, no GPU).

* the definition of every kernel the bench can report on is found in its source file: from its
  template line to the brace that closes its body, with balanced braces and no neighbouring
  definition in it;
* each DRAM-traffic record in profiles/traffic.json carries the sha256 of a kernel definition;
  a record is used only while the kernel's definition still has that hash, and editing the
  kernel (here, a copy of the source with one changed character) voids it.
"""
import hashlib
import json
import os
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("name", sorted(bench.KERNEL_SOURCE))
def test_kernel_definition_is_found_whole(name):
    text = bench.kernel_text(name)
    assert text is not None
    assert "__global__" in text and (name + "(") in text
    assert text.rstrip().endswith("}")
    assert text.count("{") == text.count("}")
    assert text.count("__global__") == 1


def test_traffic_records_follow_the_kernel_text(tmp_path, monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)["kernels"]
    assert recs
    for name, rec in recs.items():
        assert name in bench.KERNEL_SOURCE
        assert len(rec["kernel_sha256"]) == 64 and rec["dram_bytes_per_launch"]
        ok = rec["kernel_sha256"] == hashlib.sha256(bench.kernel_text(name).encode()).hexdigest()
        for wl, val in rec["dram_bytes_per_launch"].items():
            assert wl in bench.WORKLOADS and val > 0
            assert bench.traffic_for(name, wl) == (val if ok else None)
    # an edited kernel loses its record: point the bench at a copy with one changed character
    name = "tc_gemm_kernel"
    src_dir = tmp_path / "paper_2009_01054_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(
        open(os.path.join(ROOT, "profiles", "traffic.json")).read())
    src = open(os.path.join(ROOT, "paper_2009_01054_gb300", "csrc", bench.KERNEL_SOURCE[name])).read()
    text = bench.kernel_text(name)
    edited = src.replace(text, text.replace("TC_CHUNK", "TC_CHUNK ", 1))
    assert edited != src
    (src_dir / bench.KERNEL_SOURCE[name]).write_text(edited)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    for wl in bench.WORKLOADS:
        assert bench.traffic_for(name, wl) is None
