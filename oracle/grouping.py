"""Rounding of scan positions and the greedy disjoint-group schedule.

The paper updates one position after another (M-rPIE section).  The
data-parallel schedule groups positions whose W x W crop boxes are pairwise
disjoint, so that all object updates inside a group touch different pixels
and commute.  Definition used here (and by the library):

* corner_j = floor(pos_j + 0.5) per axis;
* boxes i and j overlap  <=>  |cy_i - cy_j| < W  and  |cx_i - cx_j| < W;
* positions are taken in scan order (or a caller-given permutation) and each
  goes to the FIRST existing group that has no member overlapping it (and
  fewer than ``max_group`` members when ``max_group > 0``); if there is none a
  new group is opened at the end.

``max_group = 1`` reproduces the paper's strictly sequential algorithm: one
position per group, in scan order.
"""
import numpy as np

from .model import crop_corners


def overlaps(ci, cj, W):
    """True when the W x W boxes with corners ci and cj share a pixel."""
    return abs(int(ci[0]) - int(cj[0])) < W and abs(int(ci[1]) - int(cj[1])) < W


def greedy_groups(pos, W, order=None, max_group=0):
    """Partition positions into groups of pairwise-disjoint crop boxes.

    Returns a list of int64 arrays (position indices, in placement order).
    """
    corners = crop_corners(pos)
    N = len(corners)
    order = np.arange(N) if order is None else np.asarray(order, dtype=np.int64)
    group_of = np.full(N, -1, dtype=np.int64)
    groups = []
    for n in range(len(order)):
        j = order[n]
        earlier = order[:n]
        d = np.abs(corners[earlier] - corners[j])
        clash = earlier[(d[:, 0] < W) & (d[:, 1] < W)]
        taken = set(group_of[clash].tolist())
        g = 0
        while g < len(groups) and (
            g in taken or (max_group > 0 and len(groups[g]) >= max_group)
        ):
            g += 1
        if g == len(groups):
            groups.append([])
        groups[g].append(int(j))
        group_of[j] = g
    return [np.asarray(g, dtype=np.int64) for g in groups]
