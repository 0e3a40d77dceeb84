"""Host logic of the batched form (paper_1603_09724_gb300.batch), without a GPU: the
autotuner keeps the fastest candidate per shape, writes its table to JSON and reuses it
without measuring again; shapes round N up to a multiple of 32."""
import json

from paper_1603_09724_gb300 import batch


def test_autotuner_picks_the_fastest_and_reuses_the_table(tmp_path):
    path = str(tmp_path / "tune.json")
    times = {json.dumps(c, sort_keys=True): ms for c, ms in zip(batch.CANDIDATES, (3.0, 1.5, 2.0))}
    calls = []

    def timer(c):
        calls.append(c)
        return times[json.dumps(c, sort_keys=True)]

    t = batch.Autotuner(path)
    assert t.choose("d2-m64-N64-p1", timer) == batch.CANDIDATES[1]
    assert len(calls) == len(batch.CANDIDATES)
    table = json.load(open(path))
    assert table["d2-m64-N64-p1"]["ms"] == 1.5 and len(table["d2-m64-N64-p1"]["tried"]) == 3
    t2 = batch.Autotuner(path)
    assert t2.choose("d2-m64-N64-p1", lambda c: calls.append(c) or 0.0) == batch.CANDIDATES[1]
    assert len(calls) == len(batch.CANDIDATES)


def test_shape_key_buckets_N():
    mk = lambda N, m=64: batch.Instance("k", 2, m, 10.0, None, N, 0.0, 0.0, 0.0)
    assert batch.shape_key(mk(17), 1) == batch.shape_key(mk(32), 1) == "d2-m64-N32-p1"
    assert batch.shape_key(mk(33), 1) == "d2-m64-N64-p1"
    assert batch.shape_key(mk(33, 96), 0) == "d2-m96-N64-p0"
