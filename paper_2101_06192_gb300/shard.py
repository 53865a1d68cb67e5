"""Trees split across processes, one GPU each.

The paper's distributed implementation gives each MPI rank its own share of
the tau trees and combines the ranks' u*-edge counts (Sec. 6.1, parallel
implementation).  Here a tree is a pure function of (seed, tree index), so a
rank samples the global tree range tree_range(rank, world, tau) with
fc_sample_usts(tree_offset = first tree) and the ranks sum their R and C
vectors with one all-reduce: the totals are bit-identical to a single-process
run of all tau trees, in any rank count.  The all-reduce runs through
torch.distributed (NCCL for device tensors, gloo on the CPU).
"""
from __future__ import annotations


def tree_range(rank: int, world: int, tau: int) -> tuple[int, int]:
    """(first tree, number of trees) of this rank's share of tau trees: the
    ranks hold consecutive, disjoint ranges covering [0, tau)."""
    if world < 1 or not 0 <= rank < world or tau < 0:
        raise ValueError("tree_range: need 0 <= rank < world and tau >= 0")
    lo = tau * rank // world
    hi = tau * (rank + 1) // world
    return lo, hi - lo


def allreduce_counts(*counts, group=None):
    """Sum the ranks' count vectors (R, C, fixed-point totals) in place; integer
    sums are exact, so the result does not depend on the reduction order."""
    import torch.distributed as dist
    for t in counts:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return counts
