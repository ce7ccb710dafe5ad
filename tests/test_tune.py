"""Search logic of the autotuner (CPU, fake measurements): the fastest
converging candidate wins by its median, non-converging candidates never
win, far-behind candidates are measured once, choices survive a cache round
trip."""
import pytest

from paper_2504_02117_gb300 import tune


def _fake(values, fail=(), noise=None):
    calls = []

    def measure(c):
        calls.append(c)
        k = len([x for x in calls if x == c]) - 1
        v = values[c.s] * (noise[k % len(noise)] if noise else 1.0)
        return {"value": v, "converged": c.s not in fail, "status": 0}
    return measure, calls


def test_grid_and_candidate_validation():
    g = tune.grid((1, 4), ("gmres", "bicgstab"), ("fp32", "fp64"))
    assert len(g) == 8 and g[0] == tune.Candidate(1, "gmres", "fp32", 30)
    assert len({c.key() for c in g}) == 8
    with pytest.raises(ValueError):
        tune.Candidate(0)
    with pytest.raises(ValueError):
        tune.Candidate(4, solver="lu")


def test_fastest_converging_candidate_wins_by_median():
    values = {1: 3.6e7, 2: 5.4e7, 4: 7.3e7, 8: 7.5e7, 16: 4.2e7}
    measure, calls = _fake(values, noise=(1.0, 0.9, 1.1))
    best, table = tune.autotune(measure, tune.grid(values, ("gmres",)), repeats=3, prune=0.5)
    assert best.s == 8
    assert [e["candidate"].s for e in table][:2] == [8, 4]
    assert table[0]["value"] == pytest.approx(7.5e7)          # median of 1.0, 0.9, 1.1
    assert all(len(e["values"]) == 3 for e in table if not e["pruned"])


def test_non_converging_candidate_never_wins():
    values = {1: 1.0, 2: 2.0, 4: 9.0}
    measure, _ = _fake(values, fail=(4,))
    best, table = tune.autotune(measure, tune.grid(values, ("gmres",)), repeats=2)
    assert best.s == 2
    assert table[-1]["candidate"].s == 4 and table[-1]["value"] == 0.0
    measure, _ = _fake(values, fail=(1, 2, 4))
    best, _ = tune.autotune(measure, tune.grid(values, ("gmres",)), repeats=2)
    assert best is None


def test_far_behind_candidates_are_measured_once():
    values = {1: 1.0, 2: 10.0, 4: 4.0}
    measure, calls = _fake(values)
    best, table = tune.autotune(measure, tune.grid(values, ("gmres",)), repeats=3, prune=0.5)
    assert best.s == 2
    n = {s: len([c for c in calls if c.s == s]) for s in values}
    assert n == {1: 1, 2: 3, 4: 1}
    assert {e["candidate"].s for e in table if e["pruned"]} == {1, 4}


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    c = tune.TuneCache(path)
    key = tune.TuneCache.key((128, 128, 128), 14581760, "ilu0", 1e-10, "GB300")
    assert c.get(key) is None
    cand = tune.Candidate(8, "bicgstab", "fp32", 30)
    c.put(key, cand, 8.4e7)
    again = tune.TuneCache(path)
    assert again.get(key) == cand and again.data[key]["value"] == 8.4e7


def test_inner_tolerance_follows_the_slab_readings():
    assert tune.inner_tol(8, "fp32") == 1e-2 and tune.inner_tol(2, "fp64") == 1e-2
    assert tune.inner_tol(1, "fp64") == 1e-10 and tune.inner_tol(1, "fp32") == 1e-5


def test_batch_shape_search_and_cache(tmp_path):
    """The same search over batched launch shapes: the fastest converging
    shape wins, a shape that cannot run (not converged) never does, and the
    choice survives the cache under the batch's key."""
    vals = {(1, 512): 2.7e7, (2, 512): 3.4e7, (4, 512): 4.7e7, (8, 512): 3.9e7,
            (16, 512): 2.0e7, (4, 256): 4.1e7}

    def measure(sh):
        k = (sh.cluster_ctas, sh.cta_threads)
        return {"value": vals.get(k, 0.0), "converged": k in vals}
    shapes = tune.batch_shapes((1, 2, 4, 8, 16), (512, 256))
    assert len(shapes) == 10 and shapes[0] == tune.BatchShape(1, 512)
    best, table = tune.autotune(measure, shapes, repeats=2)
    assert best == tune.BatchShape(4, 512)
    assert not any(e["converged"] for e in table if e["candidate"] == tune.BatchShape(16, 256))
    cache = tune.TuneCache(str(tmp_path / "t.json"))
    key = tune.TuneCache.batch_key([4096 * 4] * 8 + [32 ** 3 * 16], "gpu0")
    cache.put_batch(key, best, table[0]["value"])
    again = tune.TuneCache(cache.path)
    assert again.get_batch(key) == best and again.get(key) is None
    with pytest.raises(ValueError):
        tune.BatchShape(17)
    with pytest.raises(ValueError):
        tune.BatchShape(2, 384)
