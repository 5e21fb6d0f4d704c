"""Host logic of the batched launch (CPU): how groups are spread over lanes."""
import itertools

from paper_2212_01253_gb300.batch import assign_lanes


def test_every_job_lands_on_exactly_one_lane():
    costs = [5.0, 1.0, 3.0, 3.0, 2.0, 8.0, 0.5]
    out = assign_lanes(costs, 3)
    assert sorted(itertools.chain(*out)) == list(range(len(costs)))
    assert assign_lanes(costs, 1) == [[5, 0, 2, 3, 4, 1, 6]]      # one lane: longest first


def test_longest_first_balances_within_the_largest_job():
    """Greedy longest-first leaves the heaviest lane at most one job (the
    largest) above the lightest, and no worse than 4/3 of the optimum here."""
    costs = [7, 7, 6, 6, 5, 4, 4, 3, 2, 2, 1]
    out = assign_lanes(costs, 4)
    loads = [sum(costs[i] for i in lane) for lane in out]
    assert max(loads) - min(loads) <= max(costs)
    best = sum(costs) / 4
    assert max(loads) <= 4 / 3 * max(best, max(costs))


def test_more_lanes_than_jobs_leaves_lanes_empty():
    out = assign_lanes([2.0, 1.0], 4)
    assert out == [[0], [1], [], []]
