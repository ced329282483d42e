"""The peel autotuner's search logic on the CPU (fake knobs and timer; no GPU)."""
import pytest

torch = pytest.importorskip("torch")

import paper_2306_08623_gb300.nucleus as nc  # noqa: E402


def test_autotune_picks_the_fastest_pair_and_sets_it(monkeypatch):
    state = {"g": None, "t": None}
    seen = []
    monkeypatch.setattr(nc, "set_peel_max_group", lambda g: state.__setitem__("g", g))
    monkeypatch.setattr(nc, "set_peel_task_items", lambda t: state.__setitem__("t", t))
    cost = {(16, 0): 9.0, (16, -1): 7.0, (64, 0): 5.0, (64, -1): 3.0, (256, 0): 4.0, (256, -1): 6.0}

    def timer(run):
        run()
        return cost[(state["g"], state["t"])]

    res = nc.autotune_peel(lambda: seen.append((state["g"], state["t"])), max_groups=(16, 64, 256),
                           task_items=(0, -1), repeats=2, timer=timer)
    assert res["best"] == (64, -1)
    assert state == {"g": 64, "t": -1}
    assert res["times_ms"] == cost
    assert len(seen) == 12  # every pair, twice


def test_autotune_max_group_wrapper(monkeypatch):
    state = {"g": None}
    monkeypatch.setattr(nc, "set_peel_max_group", lambda g: state.__setitem__("g", g))
    monkeypatch.setattr(nc, "set_peel_task_items", lambda t: None)
    times = nc.autotune_peel_max_group(lambda: None, candidates=(4, 8, 32),
                                       timer=lambda run: {4: 2.0, 8: 1.0, 32: 1.5}[state["g"]])
    assert times == {4: 2.0, 8: 1.0, 32: 1.5}
    assert state["g"] == 8


def test_autotune_three_knobs(monkeypatch):
    state = {"g": None, "t": None, "sp": None}
    monkeypatch.setattr(nc, "set_peel_max_group", lambda g: state.__setitem__("g", g))
    monkeypatch.setattr(nc, "set_peel_task_items", lambda t: state.__setitem__("t", t))
    monkeypatch.setattr(nc, "set_relist_split", lambda sp: state.__setitem__("sp", sp))
    cost = lambda: {1: 3.0, 64: 2.0}[state["g"]] * {0.5: 1.0, 2.0: 0.5}[state["sp"]] + (state["t"] == 0)
    res = nc.autotune_peel(lambda: None, max_groups=(1, 64), task_items=(0, -1), splits=(0.5, 2.0),
                           timer=lambda run: cost())
    assert res["best"] == (64, -1, 2.0) and state == {"g": 64, "t": -1, "sp": 2.0}
    assert len(res["times_ms"]) == 8
