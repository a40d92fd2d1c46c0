"""The tune cache: its JSON format and the host-side lookup aao_create performs (no GPU).

aao_tune_lookup matches device name, dim, grid, ell and precision, prefers an entry with the
same inner iteration count, ignores keys it does not know, and refuses unreadable files.
"""
import json

import pytest

from paper_2506_03947_gb300 import binding, tune


def _entry(**kw):
    e = {"device": "GPU-A", "dim": 2, "n": [1024, 1024, 1], "ell": 10, "prec": "mixed", "p": 40,
         "kernel": "stream", "S": 4, "H": 88, "D": 3, "NW": 8, "us_per_apply": 600.0}
    e.update(kw)
    return e


def _write(tmp_path, entries, name="cache.json"):
    path = tmp_path / name
    path.write_text(json.dumps({"version": 1, "entries": entries}))
    return str(path)


def test_lookup_matches_device_grid_ell_and_precision(tmp_path):
    path = _write(tmp_path, [_entry(), _entry(device="GPU-B", H=40), _entry(n=[512, 512, 1], H=16),
                             _entry(ell=12, H=28), _entry(prec="fp64", kernel="tile")])
    look = lambda dev, n, ell, prec: binding.aao_tune_lookup(path, dev, 2, n, ell, prec, 40)
    assert look("GPU-A", (1024, 1024), 10, 1) == {"kernel": "stream", "S": 4, "H": 88, "D": 3, "NW": 8}
    assert look("GPU-B", (1024, 1024), 10, 1)["H"] == 40
    assert look("GPU-A", (512, 512), 10, 1)["H"] == 16
    assert look("GPU-A", (1024, 1024), 12, 1)["H"] == 28
    assert look("GPU-A", (1024, 1024), 10, 0)["kernel"] == "tile"
    assert look("GPU-C", (1024, 1024), 10, 1) is None
    assert look("GPU-A", (1024, 1000), 10, 1) is None
    assert look(None, (512, 512), 10, 1)["H"] == 16          # any device


def test_lookup_prefers_the_same_inner_iteration_count(tmp_path):
    path = _write(tmp_path, [_entry(p=10, H=16), _entry(p=40, H=88), _entry(p=20, H=64)])
    assert binding.aao_tune_lookup(path, "GPU-A", 2, (1024, 1024), 10, 1, 40)["H"] == 88
    assert binding.aao_tune_lookup(path, "GPU-A", 2, (1024, 1024), 10, 1, 20)["H"] == 64
    # no entry with p = 7: some matching entry is used
    assert binding.aao_tune_lookup(path, "GPU-A", 2, (1024, 1024), 10, 1, 7)["H"] in (16, 64, 88)


def test_lookup_ignores_unknown_keys_and_kernels(tmp_path):
    path = _write(tmp_path, [_entry(kernel="warp-magic", H=100), dict(_entry(H=22), note={"x": [1, 2, "y"]})])
    assert binding.aao_tune_lookup(path, "GPU-A", 2, (1024, 1024), 10, 1, 40)["H"] == 22


def test_lookup_refuses_unreadable_or_malformed_files(tmp_path):
    with pytest.raises(binding.AaoError):
        binding.aao_tune_lookup(str(tmp_path / "missing.json"), "GPU-A", 2, (64, 64), 10, 1, 40)
    bad = tmp_path / "bad.json"
    bad.write_text('{"version": 1, "entries": [{"device": "GPU-A", "n": [1, 2')
    with pytest.raises(binding.AaoError):
        binding.aao_tune_lookup(str(bad), "GPU-A", 2, (64, 64), 10, 1, 40)
    nolist = tmp_path / "nolist.json"
    nolist.write_text('{"version": 1}')
    with pytest.raises(binding.AaoError):
        binding.aao_tune_lookup(str(nolist), "GPU-A", 2, (64, 64), 10, 1, 40)


def test_save_entry_replaces_the_same_key_and_round_trips(tmp_path):
    path = str(tmp_path / "c.json")
    tune.save_entry(path, _entry(H=16))
    tune.save_entry(path, _entry(device="GPU-B"))
    tune.save_entry(path, _entry(H=64))                        # same key as the first: replaced
    d = tune.load(path)
    assert len(d["entries"]) == 2
    assert binding.aao_tune_lookup(path, "GPU-A", 2, (1024, 1024), 10, 1, 40)["H"] == 64
    e = tune.make_entry("GPU-A", 2, (1024, 1024), 10, binding.AAO_MIXED, 40,
                        {"kernel": "stream", "S": 2, "H": 58, "D": 4, "NW": 12, "us_per_apply": 1.5})
    assert e["n"] == [1024, 1024, 1] and e["prec"] == "mixed" and e["S"] == 2
