"""Host-side logic of the batched launch (no GPU): the stream plan and the seeded instance mix."""
import numpy as np
import pytest

from paper_2012_05537_gb300 import build as B
from paper_2012_05537_gb300 import inputs as I


@pytest.fixture(scope="module")
def S():
    B.build()
    from paper_2012_05537_gb300 import sllbm
    sllbm.load()
    return sllbm


def test_plan_is_longest_processing_time_first(S):
    # sorted 5,4,3,3,2,2,1 onto 3 streams: loads 5 | 4 | 3 -> 3 to the 3-stream (6), 2 to the
    # 4-stream (6), 2 to the 5-stream (7), 1 to the lowest-index least-loaded stream (1)
    assert list(S.sllbm_batch_plan([5, 4, 3, 3, 2, 2, 1], 3)) == [0, 1, 2, 2, 1, 0, 1]
    assert list(S.sllbm_batch_plan([1.0], 4)) == [0]
    assert list(S.sllbm_batch_plan([2, 2, 2, 2], 2)) == [0, 1, 0, 1]


def test_plan_balances_random_costs(S):
    cost = I.rng(3).uniform(0.0, 1.0, 200)
    assign = S.sllbm_batch_plan(cost, 8)
    loads = np.bincount(assign, weights=cost, minlength=8)
    # LPT bound: max load <= mean load + largest job
    assert loads.max() <= loads.mean() + cost.max() + 1e-12


def test_plan_rejects_bad_arguments(S):
    for args in (([1.0, -1.0], 2), ([1.0], 0)):
        with pytest.raises(S.SllbmError):
            S.sllbm_batch_plan(*args)


def test_batch_instances_are_seeded_and_in_range():
    a, b = I.batch_instances(64, 0), I.batch_instances(64, 0)
    assert a == b and a != I.batch_instances(64, 1)
    for inst in a:
        n = inst.cells[0]
        assert inst.cells == (n, n, n) and 8 <= n <= 24 and inst.p in (2, 3, 4)
        assert 0.3 <= inst.Ma <= 1.25 and 400 <= inst.Re <= 1600 and 1 <= inst.courant <= 8
    assert {inst.p for inst in a} == {2, 3, 4}
