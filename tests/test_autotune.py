"""Host logic of the autotuner: picks the fastest candidate, skips failing
ones, caches by signature (no GPU needed: the simulator is faked)."""
import json

import pytest

from paper_2103_00081_gb300 import autotune as AT


class FakeSim:
    def __init__(self, opts, times):
        self.opts = opts
        self.times = times

    def step(self, dt, check=True):
        if self.opts.get("broken"):
            return {"rc": -4, "ms_total": 0.0}
        return {"rc": 0, "ms_total": self.times[self.opts["id"]]}

    def close(self):
        pass


def test_tune_picks_fastest_and_caches(tmp_path):
    times = {0: 5.0, 1: 2.0, 2: 3.0}
    cands = [{"id": 0}, {"id": 1}, {"id": 2}, {"id": 3, "broken": True}]
    cache = str(tmp_path / "c.json")
    best, table = AT.tune(lambda o: FakeSim(o, times), 1.0, "sig", cands, steps=2, cache=cache)
    assert best == {"id": 1}
    assert [t[1] for t in table[:3]] == [5.0, 2.0, 3.0]
    assert table[3][2].startswith("failed")
    data = json.load(open(cache))
    assert data["sig"]["opts"] == {"id": 1}
    # cached: a different timing table is ignored unless forced
    best2, _ = AT.tune(lambda o: FakeSim(o, {0: 1.0, 1: 9.0, 2: 9.0}), 1.0, "sig", cands, cache=cache)
    assert best2 == {"id": 1}
    best3, _ = AT.tune(lambda o: FakeSim(o, {0: 1.0, 1: 9.0, 2: 9.0}), 1.0, "sig", cands[:3], cache=cache,
                       force=True)
    assert best3 == {"id": 0}


def test_tune_raises_when_everything_fails(tmp_path):
    with pytest.raises(RuntimeError):
        AT.tune(lambda o: FakeSim(o, {}), 1.0, "s", [{"broken": True}], cache=None)


class FakeBatch:
    def __init__(self, opts, delay):
        self.opts = opts
        self.delay = delay

    def step(self, dt, check=True):
        import time
        time.sleep(self.delay[self.opts["planes"]])
        rc = -6 if self.opts["planes"] == 99 else 0
        return [{"rc": rc}, {"rc": 0}]

    def close(self):
        pass


def test_tune_batch_times_whole_batched_steps(tmp_path):
    delay = {0: 0.03, 8: 0.005, 16: 0.02, 99: 0.0}
    cands = [{"mode": 2, "planes": p} for p in (0, 8, 16, 99)]
    best, table = AT.tune_batch(lambda o: FakeBatch(o, delay), 1.0, "b", cands, steps=1,
                                cache=str(tmp_path / "c.json"))
    assert best == {"mode": 2, "planes": 8}
    assert table[3][2].startswith("failed")       # a step that returned an error
    assert table[0][1] > table[1][1]
    assert all(c["mode"] in (0, 2) for c in AT.default_batch_candidates())
