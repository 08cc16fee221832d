"""Host-side logic of the benchmark that needs no GPU: the traffic record's
source digest, the compact formatting of the final line and the headline's
candidate forms."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


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


def test_compact_rounding():
    assert bench.sig(1.23456789) == 1.235
    assert bench.sig({"a": [2.0 / 3.0, 7]}) == {"a": [0.6667, 7]}
    assert bench.sig(float("nan")) is None


def test_headline_forms_and_oracle_knobs():
    import oracle
    names = [f[0] for f in bench.HEAD_FORMS]
    assert len(set(names)) == len(names)
    for f in bench.HEAD_FORMS:
        k = bench.form_oracle_knobs(oracle, f, 8)
        assert k.mode == f[1] and (k.st[0] is not None) == f[2]
