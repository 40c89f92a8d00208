"""Pins of the disjoint-group schedule: pairwise disjointness, and equality with
an independently written group-by-group greedy construction (which yields the
same partition as first-fit by position)."""
import numpy as np
import pytest

from oracle import grouping, model


def group_by_group(pos, W, max_group=0):
    """Build group 0 by scanning all positions in order and taking each one
    that fits, then group 1 from what is left, and so on."""
    c = model.crop_corners(pos)
    left = list(range(len(c)))
    groups = []
    while left:
        g, rest = [], []
        for j in left:
            full = max_group > 0 and len(g) >= max_group
            if not full and all(not (abs(c[i][0] - c[j][0]) < W and abs(c[i][1] - c[j][1]) < W) for i in g):
                g.append(j)
            else:
                rest.append(j)
        groups.append(g)
        left = rest
    return groups


@pytest.mark.parametrize("seed,W,mg", [(0, 8, 0), (1, 16, 0), (2, 8, 3), (3, 5, 0)])
def test_groups_equal_group_by_group_greedy(seed, W, mg):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 40, size=(120, 2))
    got = grouping.greedy_groups(pos, W, max_group=mg)
    ref = group_by_group(pos, W, mg)
    assert [list(g) for g in got] == ref
    c = model.crop_corners(pos)
    seen = np.concatenate(got)
    assert sorted(seen.tolist()) == list(range(len(pos)))
    for g in got:
        for a in range(len(g)):
            for b in range(a + 1, len(g)):
                assert not grouping.overlaps(c[g[a]], c[g[b]], W)


def test_sequential_groups_and_permutation():
    pos = np.random.default_rng(5).uniform(0, 30, size=(20, 2))
    gs = grouping.greedy_groups(pos, 8, max_group=1)
    assert [g.tolist() for g in gs] == [[j] for j in range(20)]
    order = np.random.default_rng(6).permutation(20)
    gs = grouping.greedy_groups(pos, 8, order=order, max_group=1)
    assert [g.tolist() for g in gs] == [[int(j)] for j in order]


def test_boundary_touching_boxes_are_disjoint():
    pos = np.array([[0.0, 0.0], [0.0, 8.0], [7.0, 7.0], [8.0, 0.0]])
    gs = grouping.greedy_groups(pos, 8)
    assert [g.tolist() for g in gs] == [[0, 1, 3], [2]]
