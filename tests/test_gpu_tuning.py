"""The autotuner's choices persist as JSON lines keyed by GPU, dataset shape
and batch shape, and come back into a new dataset (explicitly, or through
GGEVAL_TUNE_CACHE during ggeval_autotune)."""
import json
import os
import time

import pytest
import torch

import parity as PA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_30954_gb300 as pkg
    pkg.lib()
    return pkg


def test_tuning_file_round_trip(gg, tmp_path, monkeypatch):
    w = PA.build("c2", 40_000, 512)
    X, y = torch.from_numpy(w["X"]), torch.from_numpy(w["y"])
    op, cv = torch.from_numpy(w["op"]).cuda(), torch.from_numpy(w["cval"]).cuda()
    ds = gg.Dataset(X, y)
    ds.autotune(op, cv)
    chosen = ds.tile_config(op, cv)
    path = str(tmp_path / "tune.jsonl")
    ds.tuning_save(path)
    rows = [json.loads(line) for line in open(path)]
    assert len(rows) == 1 and rows[0]["trials"] == 512 and rows[0]["rows"] == 40_000
    assert (rows[0]["variant"], rows[0]["tile_rows"], rows[0]["group"], rows[0]["warps"]) == chosen
    ref = ds.eval_batch(op, cv)[0].clone()
    ds.sync()
    ds.close()
    # a new dataset takes the entry back
    ds2 = gg.Dataset(X, y)
    assert ds2.tuning_load(path) == 1
    assert ds2.tile_config(op, cv) == chosen
    got = ds2.eval_batch(op, cv)[0]
    ds2.sync()
    assert torch.equal(ref, got)
    ds2.close()
    # through the environment: autotune finds the entry and times nothing
    monkeypatch.setenv("GGEVAL_TUNE_CACHE", path)
    ds3 = gg.Dataset(X, y)
    t0 = time.perf_counter()
    ds3.autotune(op, cv)
    assert time.perf_counter() - t0 < 0.5
    assert ds3.tile_config(op, cv) == chosen
    # another batch shape is tuned and appended
    ds3.autotune(op[:256].contiguous(), cv[:256].contiguous())
    assert len(open(path).read().splitlines()) == 2
    ds3.close()
    # a dataset of another shape takes nothing
    ds4 = gg.Dataset(X[:30_000].contiguous(), y[:30_000].contiguous())
    assert ds4.tuning_load(path) == 0
    ds4.close()
