"""Host-side pieces of the benchmark that set its CPU baseline: the pair count of
sampled targets (the numerator of the oracle's throughput) and the oracle pool.

The vectorised count (per-box neighbourhood sizes minus the target itself) must
equal the per-target count that also removes coincident points, on a point set
without duplicates, and fall back to it when duplicates exist.
"""
import numpy as np

import bench
import oracle
from paper_2403_01596_gb300 import workloads as W


def _structure(points, lo, h, ng):
    b = oracle.bin_points(points, lo, h, ng)
    nptr, nidx = oracle.neighbors(b["box_keys"], ng)
    return (b["box_ptr"], nptr, nidx, b["point_box"], b["perm"])


def test_sample_pairs_fast_matches_exact_count():
    pts = W.unit_sphere(20000, 31)
    st = _structure(pts, (-1.0, -1.0, -1.0), 2.0 / 24, 24)
    targets = bench._sample_targets(len(pts), 700, 5)
    assert bench._sample_pairs_fast(st, pts, targets) == bench._sample_pairs(st, pts, targets)
    # the sampled count summed over every target is the oracle's own pair count
    all_t = np.arange(len(pts))
    assert bench._sample_pairs_fast(st, pts, all_t) == oracle.pair_count(pts, (-1.0, -1.0, -1.0), 2.0 / 24, 24)


def test_sample_pairs_fast_with_duplicates_falls_back():
    pts = W.uniform_cube(3000, 32)
    pts = np.concatenate([pts, pts[:50]])  # 50 coincident pairs: r = 0 skipped for both
    st = _structure(pts, (0.0, 0.0, 0.0), 0.25, 4)
    targets = np.arange(len(pts))
    n = bench._sample_pairs_fast(st, pts, targets)
    assert n == bench._sample_pairs(st, pts, targets)
    assert n == oracle.pair_count(pts, (0.0, 0.0, 0.0), 0.25, 4)


def test_oracle_pool_times_shares_and_closes():
    """Two spawned oracle workers: each rebuilds the seeded sweep workloads, runs its share behind a barrier,
    and the pool shuts down cleanly."""
    pool = bench.OraclePool(workers=2)
    try:
        assert pool.workers == 2
        targets = bench._sample_targets(1 << 20, 64, 3)
        dt = pool.run(3, targets)  # occupancy 64, 32 targets per worker
        assert 0.0 < dt < 120.0
        assert all(pr.is_alive() for pr in pool.procs)
    finally:
        pool.close()
    assert not any(pr.is_alive() for pr in pool.procs)
