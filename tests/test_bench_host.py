"""Host logic of bench.py's CPU legs (no GPU): the in-cutoff pair count that the oracle's
throughput is divided by, against the oracle's brute-force pair set."""
import numpy as np

import oracle
from paper_2503_20541_b300 import workloads as wl


def test_cutoff_pair_count_matches_the_oracle_pair_set():
    import bench
    s = wl.water_box_density(400, seed=3)
    x = s.x.astype(np.float64)
    p = oracle.make_params(s.box, r_cut=s.r_cut)
    pairs, _ = oracle.neighbor_pairs(x, p, s.r_cut, excl=s.excl)
    assert bench.cutoff_pairs_kdtree(s) == len(pairs)
