"""The throughput the benchmark reports is the paper's: grid cells x time steps / time
(Table 1).  The three printed rows pin the definition."""
import os

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def test_table1_rows_reproduce_with_bench_metric():
    rows = [l for l in open(os.path.join(HERE, "golden", "table1_gcells.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        _, _, n, steps, t, g = [c.strip() for c in r.split("|")]
        got = bench.gpts_per_s(int(n) ** 3, int(steps), float(t))
        assert round(got, 2) == float(g), (r, got)
