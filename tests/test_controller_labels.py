"""The labelling search of the learned (q, p) controller (host logic, no GPU).

`controller_train.label` returns the fastest (q, p) of the grid whose rSVD
meets the target, timing only the smallest passing p of each q.  Here the
rSVD, its residual and its timing are replaced by a table, and the search is
checked against the exhaustive minimum over the grid: it must pick the same
configuration whenever accuracy grows with q and p and time grows with both,
stop once p = 2 passes, and fall back to (Q_MAX, P_MAX) when nothing passes.
"""
import itertools

import pytest

from paper_1608_02148_gb300 import controller_train as ct


class _Info:
    status = 0


def _install(monkeypatch, passes, cost):
    """passes(q, p) -> bool, cost(q, p) -> ms; records the calls."""
    calls = {"run": [], "timed": []}

    def run(h, A, k, p, q, seed, mode="fixed"):
        calls["run"].append((q, p))
        return (q, p), None, None, _Info()

    def residual(A, d, U, V):
        q, p = d
        return 0.0 if passes(q, p) else 1.0

    def timed(h, A, k, p, q, seed, reps=2):
        calls["timed"].append((q, p))
        return cost(q, p)

    monkeypatch.setattr(ct, "run", run)
    monkeypatch.setattr(ct, "residual", residual)
    monkeypatch.setattr(ct, "timed", timed)
    return calls


def _exhaustive(passes, cost):
    ok = [(cost(q, p), q, p) for q in ct.Q_GRID for p in ct.P_GRID if passes(q, p)]
    return min(ok)[1:] if ok else (ct.Q_MAX, ct.P_MAX)


# monotone worlds: the smallest passing p falls as q grows
_NEEDS = [
    {0: 10, 1: 6, 2: 2},          # the fastest is q = 2, p = 2 or earlier, depending on the cost
    {0: None, 1: 10, 2: 4, 3: 2},  # q = 0 never passes
    {0: 2},                        # the sketch alone is enough
    {0: None, 1: None, 2: None, 3: None, 4: None, 5: None, 6: 10},
]


@pytest.mark.parametrize("needs", _NEEDS)
@pytest.mark.parametrize("pass_ms,col_ms", [(1.0, 0.01), (0.1, 0.05), (0.02, 0.2)])
def test_label_is_the_fastest_passing_configuration(monkeypatch, needs, pass_ms, col_ms):
    def p_needed(q):
        best = None
        for qq in sorted(needs):
            if qq <= q and needs[qq] is not None:
                best = needs[qq] if best is None else min(best, needs[qq])
        return best

    def passes(q, p):
        need = p_needed(q)
        return need is not None and p >= need

    def cost(q, p):  # (2q + 2) passes plus a cost that grows with the width
        return (2 * q + 2) * pass_ms + (20 + p) * col_ms

    calls = _install(monkeypatch, passes, cost)
    q, p, runs = ct.label(None, None, 20, 0.5, 0)
    assert (q, p) == _exhaustive(passes, cost), (q, p, calls)
    assert runs == len(calls["run"]) + 2 * len(calls["timed"])
    # only the smallest passing p of a q is timed, and the search stops at p = 2
    for tq, tp in calls["timed"]:
        assert passes(tq, tp) and all(not passes(tq, x) for x in ct.P_GRID if x < tp)
    if any(tp == ct.P_GRID[0] for _, tp in calls["timed"]):
        last_q = max(tq for tq, _ in calls["timed"])
        assert all(rq <= last_q for rq, _ in calls["run"])


def test_label_falls_back_when_nothing_passes(monkeypatch):
    calls = _install(monkeypatch, lambda q, p: False, lambda q, p: 1.0)
    q, p, runs = ct.label(None, None, 20, 0.5, 0)
    assert (q, p) == (ct.Q_MAX, ct.P_MAX)
    assert calls["timed"] == []
    assert sorted(calls["run"]) == sorted(itertools.product(ct.Q_GRID, ct.P_GRID))
    assert runs == len(ct.Q_GRID) * len(ct.P_GRID)
