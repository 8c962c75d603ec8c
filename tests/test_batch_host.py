"""Host logic of the batched sweep (no GPU): the schedules the autotuner
times and its cache."""
import json

from paper_1810_04597_gb300 import batch


def test_candidates_cover_every_schedule():
    tiles, queue = (128, 256, 512, 1024), (True, False)
    c = batch.candidates(16, 8, tiles, queue)
    assert len(c) == len(set(c))
    modes = {m for _, _, _, m, _ in c}
    assert modes == {batch.PERSISTENT, batch.PHASED, batch.RUN_MAJOR}
    pers = [x for x in c if x[3] == batch.PERSISTENT]
    assert {x[0] for x in pers} == set(tiles) and {x[2] for x in pers} == set(queue)
    assert {x[1] for x in pers} == {2, 3, 4, 8}
    assert [x[4] for x in c if x[3] == batch.RUN_MAJOR] == [1, 2, 4, 8, 16]
    assert all(1 <= x[1] <= 8 for x in c)


def test_candidates_respect_limits():
    # one block per SM, three runs: no blocks-per-SM choice above the limit,
    # no more graph branches than runs
    c = batch.candidates(3, 1)
    assert all(x[1] == 1 for x in c)
    assert [x[4] for x in c if x[3] == batch.RUN_MAJOR] == [1, 2, 3]


def test_high_order_batches_run_major_only():
    c = batch.candidates(5, 4, high_order=True)
    assert c and all(x[3] == batch.RUN_MAJOR for x in c)


def test_cache_reads_missing_or_corrupt_as_empty(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setattr(batch, "TUNE_CACHE", str(path))
    assert batch._load_cache() == {}
    path.write_text("{not json")
    assert batch._load_cache() == {}
    path.write_text(json.dumps({"k": {"tile": 256}}))
    assert batch._load_cache() == {"k": {"tile": 256}}
