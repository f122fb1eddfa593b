"""Host-side helpers of the learned-schedule measurement, against closed forms:
rank correlation, greedy list-scheduling makespan (the persistent queue's
behaviour) and the degree-bucket schedule's wedge-work estimate."""
import numpy as np
import pytest

from paper_1911_10616_gb300 import graphgen as gg

learned = pytest.importorskip("paper_1911_10616_gb300.learned")


def test_spearman_closed_forms():
    a = np.arange(50.0)
    assert learned.spearman(a, a ** 3) == pytest.approx(1.0)
    assert learned.spearman(a, -a) == pytest.approx(-1.0)
    # textbook value: rho = 1 - 6 sum d^2 / (n (n^2 - 1)) for distinct ranks
    x = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    y = np.array([2.0, 1.0, 4.0, 3.0, 5.0])
    assert learned.spearman(x, y) == pytest.approx(1 - 6 * 4 / (5 * 24))


def test_list_schedule_makespan():
    c = np.array([5.0, 3.0, 3.0, 2.0, 2.0, 1.0])
    assert learned.list_schedule_makespan(c, range(6), 1) == c.sum()
    assert learned.list_schedule_makespan(c, range(6), 6) == c.max()
    # two workers, longest first: {5, 2, 1} and {3, 3, 2} -> 8
    assert learned.list_schedule_makespan(c, np.argsort(-c, kind="stable"), 2) == 8.0
    # the bad order the learned model is compared against: shortest first
    # A: 1, 2, 3 -> 6; B: 2, 3, 5 -> 10
    assert learned.list_schedule_makespan(c, np.argsort(c, kind="stable"), 2) == 10.0


def test_wedge_work_is_sum_of_neighbour_degrees():
    g = gg.chung_lu(2000, 8000, 2.1, 80, 3)
    d = g.degrees()
    want = np.array([d[g.col[g.rowptr[u]:g.rowptr[u + 1]]].sum() for u in range(g.n)])
    assert np.array_equal(learned.wedge_work(g).astype(np.int64), want)
