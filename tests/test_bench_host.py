"""Host logic of bench.py that needs no GPU: the kernel-source hash that ties the
committed ncu traffic figures to the sources they were measured on."""
import json
import os

import bench


def _tree(root, with_cache):
    csrc = os.path.join(root, "paper_2110_01585_gb300", "csrc")
    os.makedirs(csrc)
    with open(os.path.join(csrc, "a.cu"), "w") as f:
        f.write("// kernel a\n")
    with open(os.path.join(csrc, "b.cuh"), "w") as f:
        f.write("// header b\n")
    if with_cache:
        os.makedirs(os.path.join(csrc, "__pycache__"))
        with open(os.path.join(csrc, "__pycache__", "gen.cpython-312.pyc"), "wb") as f:
            f.write(b"\x00\x01")
    return csrc


def test_source_hash_ignores_bytecode_caches(tmp_path, monkeypatch):
    _tree(str(tmp_path / "clean"), with_cache=False)
    _tree(str(tmp_path / "cached"), with_cache=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "clean"))
    h_clean = bench._kernel_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "cached"))
    assert bench._kernel_source_hash() == h_clean


def test_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    csrc = _tree(str(tmp_path), with_cache=False)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    os.makedirs(tmp_path / "profiles")
    entry = {"dram_bytes_per_unit": 12.5, "source_hash": bench._kernel_source_hash()}
    with open(tmp_path / "profiles" / "ncu_traffic.json", "w") as f:
        json.dump({"prior_sweep": entry}, f)
    assert bench._ncu_traffic("prior_sweep") == 12.5
    assert bench._ncu_traffic("cg_precond") is None
    with open(os.path.join(csrc, "a.cu"), "a") as f:  # the kernel changes: figure void
        f.write("// edited\n")
    assert bench._ncu_traffic("prior_sweep") is None
