"""Host-side logic of the benchmark that needs no GPU: the surrogate's
calibrated price floor and the traffic record's source digest."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_calibrated_floor_with_exact_predictions_is_the_smallest_price():
    rng = np.random.default_rng(3)
    exact = rng.uniform(0.5, 50.0, 5000)
    assert bench.calibrate_floor(exact.copy(), exact) == exact.min()


def test_calibrated_floor_stops_where_the_error_grows():
    # relative error 0.1% above a price of 10, 5% below it: the floor is the
    # smallest prediction of a prefix whose 99th percentile stays within 1%,
    # so it may not reach far below 10
    rng = np.random.default_rng(4)
    exact = rng.uniform(1.0, 20.0, 20000)
    rel = np.where(exact >= 10.0, 1e-3, 5e-2)
    pred = exact * (1.0 + rel)
    tau = bench.calibrate_floor(pred, exact)
    above = pred >= tau
    err = np.abs(pred - exact) / exact
    assert np.quantile(err[above], 0.99) <= 0.01
    assert 9.0 < tau < 11.0


def test_calibrated_floor_is_infinite_when_nothing_qualifies():
    exact = np.linspace(1.0, 2.0, 1000)
    assert bench.calibrate_floor(exact * 1.5, exact) == float("inf")


def test_traffic_record_matches_the_current_element_kernel_source():
    # the committed DRAM-bytes record is only reported while its digest equals
    # the kernel source's; a stale record reads as null
    rec = {}
    for line in open(os.path.join(bench.ROOT, "profiles", "dram_traffic.txt")):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#"):
            rec[f[0]] = f[2]
    assert set(rec) >= {"elem_kernel", "node_kernel"}
    for tag, dig in rec.items():
        assert (bench.dram_traffic(tag, 1) is not None) == (dig == bench.source_digest(tag))
