"""Host logic of the sweep-schedule autotuner, without a GPU.

The native calls the tuner makes (block count, set schedule, timed regularisation) are
replaced by a fake whose per-schedule timings are fixed, so the choice, the skipping of
schedules the library refuses and the cache can be checked on the CPU."""

import types

import pytest

from paper_1604_03734_gb300 import autotune as AT
from paper_1604_03734_gb300 import native


def test_candidates_are_distinct_and_within_the_schedule_ranges():
    cands = AT.DEFAULT_CANDIDATES
    assert len(set(cands)) == len(cands)
    for k, order, ctas, graph in cands:
        # the ranges denser_set_schedule accepts
        assert 0 <= k <= 9 and order in (0, 1) and 0 <= ctas <= 8 and graph in (0, 1)
    assert {c[0] for c in cands} == set(range(10))
    assert (7, 0, 2, 1) in cands  # the library's default schedule


class _Fake:
    def __init__(self, times, refused=(), n_blocks=24176):
        self.times, self.refused, self.n_blocks = times, set(refused), n_blocks
        self.current = None
        self.timed = []

    def install(self, monkeypatch):
        monkeypatch.setattr(AT.N, "denser_num_blocks", lambda ctx: self.n_blocks)
        monkeypatch.setattr(AT.N, "denser_set_schedule", self.set_schedule)
        monkeypatch.setattr(AT.N, "denser_regularize", self.regularize)

    def set_schedule(self, ctx, *sch):
        if tuple(sch) in self.refused:
            raise native.DenserError(native.DENSER_ERR_INVALID_ARG, "set_schedule: field out of range")
        self.current = tuple(sch)

    def regularize(self, ctx, iters, gap_tol, start, stream):
        self.timed.append(self.current)
        return types.SimpleNamespace(sweep_ms=self.times[self.current] * iters, iters=iters)


@pytest.fixture(autouse=True)
def _empty_cache(monkeypatch):
    monkeypatch.setattr(AT, "_cache", {})


def test_picks_the_fastest_and_skips_refused_schedules(monkeypatch):
    cands = [(7, 0, 2, 1), (8, 0, 2, 1), (2, 1, 0, 1), (4, 0, 9, 1)]
    fake = _Fake({(7, 0, 2, 1): 0.11, (8, 0, 2, 1): 0.10, (2, 1, 0, 1): 0.13}, refused=[(4, 0, 9, 1)])
    fake.install(monkeypatch)
    res = AT.autotune(None, precision=1, iters=10, candidates=cands)
    assert res["schedule"] == [8, 0, 2, 1] and not res["cached"]
    assert res["ms_per_iter"] == pytest.approx(0.10)
    assert [s for s, _ in res["table"]] == [[7, 0, 2, 1], [8, 0, 2, 1], [2, 1, 0, 1]]
    assert fake.current == (8, 0, 2, 1)  # the winner is left set on the context
    # one warm-up and two timed calls per schedule the library accepted
    assert len(fake.timed) == 3 * 3


def test_cache_hit_sets_the_schedule_without_timing(monkeypatch, tmp_path):
    cands = [(7, 0, 2, 1), (8, 0, 2, 1)]
    fake = _Fake({(7, 0, 2, 1): 0.09, (8, 0, 2, 1): 0.10})
    fake.install(monkeypatch)
    cache = str(tmp_path / "tune.json")
    first = AT.autotune(None, precision=0, candidates=cands, cache_file=cache)
    n_timed = len(fake.timed)
    fake.current = None
    again = AT.autotune(None, precision=0, candidates=cands, cache_file=cache)
    assert again["cached"] and again["schedule"] == first["schedule"] == [7, 0, 2, 1]
    assert len(fake.timed) == n_timed and fake.current == (7, 0, 2, 1)
    # another storage precision, or a map of another size class, is tuned afresh
    AT.autotune(None, precision=2, candidates=cands, cache_file=cache)
    assert len(fake.timed) == 2 * n_timed
    # a fresh process reads the cache file
    monkeypatch.setattr(AT, "_cache", {})
    fake.current = None
    from_file = AT.autotune(None, precision=0, candidates=cands, cache_file=cache)
    assert from_file["cached"] and fake.current == (7, 0, 2, 1) and len(fake.timed) == 2 * n_timed


def test_no_schedule_accepted_is_an_error(monkeypatch):
    fake = _Fake({}, refused=[(7, 0, 2, 1)])
    fake.install(monkeypatch)
    with pytest.raises(RuntimeError):
        AT.autotune(None, candidates=[(7, 0, 2, 1)])


def test_size_buckets_split_by_half_octaves():
    assert AT._bucket(0) == 0
    assert AT._bucket(24176) == AT._bucket(24000)
    assert AT._bucket(24176) < AT._bucket(207020) < AT._bucket(3946914)
