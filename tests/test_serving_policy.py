"""Host logic of the serving loop's batch policy (no GPU): shortest
remaining work first, filled to a minimum pack count, with a bound on how
long a request may wait for a step."""
from types import SimpleNamespace

from paper_2609_31258_b300.serving import srpt_batch


def _req(n_packs, n_steps):
    return SimpleNamespace(n_packs=n_packs, n_steps=n_steps)


def test_shortest_remaining_first_until_filled():
    active = {0: _req(1000, 100), 1: _req(10, 100), 2: _req(500, 100), 3: _req(50, 100)}
    clock = {0: 0, 1: 0, 2: 0, 3: 0}
    assert srpt_batch(active, clock, min_packs=1) == [1]
    assert srpt_batch(active, clock, min_packs=60) == [1, 3]
    assert srpt_batch(active, clock, min_packs=61) == [1, 3, 2]
    assert srpt_batch(active, clock, min_packs=10 ** 9) == [1, 3, 2, 0]


def test_remaining_work_counts_progress_and_ties_break_by_slot():
    active = {0: _req(100, 1000), 1: _req(100, 1000), 2: _req(400, 1000)}
    # slot 2 has 50 micro steps left: 400 x 50 < 100 x 1000
    clock = {0: 0, 1: 0, 2: 950}
    assert srpt_batch(active, clock, min_packs=1) == [2]
    clock = {0: 0, 1: 0, 2: 0}
    assert srpt_batch(active, clock, min_packs=150) == [0, 1]


def test_waiting_requests_are_not_starved():
    active = {0: _req(10, 100), 1: _req(10 ** 6, 100)}
    clock = {0: 0, 1: 0}
    assert srpt_batch(active, clock, 1, waited={0: 0.0, 1: 1.0}, max_defer=5.0) == [0]
    assert srpt_batch(active, clock, 1, waited={0: 0.0, 1: 6.0}, max_defer=5.0) == [0, 1]
