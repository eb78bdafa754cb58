"""Multi-process sharding of one survey (one process per GPU).

Every rank holds a replica of G+ and surveys the pivots of its own range of
the <+ order; the uint64 tables are then summed once across ranks -- the
all_reduce that closes the paper's triangle count (Alg. 2).  The ranges come
from tripoll_partition_pivots (near-equal wedge counts per range).
"""
from __future__ import annotations


def shard_range(bounds, rank: int):
    """Pivot range [lo, hi) of `rank` from partition bounds (len = world + 1)."""
    return int(bounds[rank]), int(bounds[rank + 1])


def sharded_survey(survey_range, bounds, rank: int, out, all_reduce):
    """Survey this rank's pivot range into `out`, then sum `out` across ranks.

    survey_range(lo, hi, out) writes the partial tables of pivots [lo, hi);
    all_reduce(out) sums `out` elementwise over all ranks in place."""
    lo, hi = shard_range(bounds, rank)
    survey_range(lo, hi, out)
    all_reduce(out)
    return out
