"""The sweep's schedule search (coordinate descent over the 90-point schedule
grid) on synthetic cost functions, without a GPU."""
import itertools

from paper_2308_16877_gb300 import autotune as A


def test_finds_the_optimum_of_a_separable_cost_with_few_evaluations():
    # a bowl in each coordinate (index distance from a chosen optimum)
    opt = (256, 12, 2)
    idx = [{v: i for i, v in enumerate(ax)} for ax in A.AXES]
    cost = lambda p: sum((idx[k][p[k]] - idx[k][opt[k]]) ** 2 for k in range(3)) + 1.0
    best, seen = A.coordinate_descent(cost)
    assert best == opt
    assert len(seen) < 30 < len(list(itertools.product(*A.AXES)))


def test_interacting_coordinates_end_at_a_coordinatewise_minimum():
    # the best tile size depends on the block count (a ridge along
    # blocks x tiles = 32): the search ends where no single coordinate
    # improves, having cycled at least once more after its last move
    def cost(p):
        bt, bps, tb = p
        return abs(bps * tb - 32) + 0.1 * abs(bt - 128) / 64 + 0.01 * tb
    best, seen = A.coordinate_descent(cost)
    for ax, values in enumerate(A.AXES):
        for v in values:
            q = best[:ax] + (v,) + best[ax + 1:]
            assert cost(q) >= cost(best)
            assert q in seen
    assert cost(best) <= cost(A.START)


def test_every_point_is_timed_at_most_once():
    calls = []
    A.coordinate_descent(lambda p: calls.append(p) or float(sum(p)))
    assert len(calls) == len(set(calls))
