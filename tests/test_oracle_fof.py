"""Pins of oracle.fof (Sec. 3.2 friends-of-friends): the integer linking rule at the linking
length, transitivity along chains, the periodic minimum image, the nmin cut and labels, and a
cross-check of the brute-force pair search against an independent cell-list search."""
import numpy as np
import pytest

from oracle import fof

S = 3 * 2**16          # mean separation in fixed units (ng / np = 3, F = 16)
PERIOD = 96 * 2**16    # ng 2^F for ng = 96


def coords(points):
    return np.array(points, dtype=np.int64).T


def test_linking_length_is_a_strict_integer_threshold():
    # 25 d^2 < s^2  <=>  d < s / 5; s / 5 = 39321.6 fixed units
    f = coords([[0, 0, 0], [39321, 0, 0], [78642, 0, 0], [78642 + 39322, 0, 0]])
    i, j = fof.friend_pairs(f, PERIOD, S)
    assert sorted(zip(i.tolist(), j.tolist())) == [(0, 1), (1, 2)]  # 39321 links, 39322 does not
    g, size = fof.fof_groups(f, PERIOD, S, nmin=2)
    assert g.tolist() == [0, 0, 0, -1] and size.tolist() == [3, 3, 3, 1]


def test_chain_is_one_group_and_pairs_are_not_transitive():
    step = 30000
    f = coords([[k * step, 0, 0] for k in range(10)] + [[0, 10**7, 0]])
    g, size = fof.fof_groups(f, PERIOD, S, nmin=5)
    assert g.tolist() == [0] * 10 + [-1]
    i, j = fof.friend_pairs(f, PERIOD, S)
    assert len(i) == 9  # only neighbours along the chain are friends


def test_minimum_image_across_the_box_face():
    f = coords([[5, 7, 9], [PERIOD - 5, 7, 9], [PERIOD // 2, 0, 0]])
    g, size = fof.fof_groups(f, PERIOD, S, nmin=2)
    assert g.tolist() == [0, 0, -1]


def test_labels_are_the_smallest_member_index():
    rng = np.random.default_rng(3)
    f = rng.integers(0, PERIOD, size=(3, 400))
    f[:, 200:260] = f[:, 199:200] + rng.integers(-8000, 8000, size=(3, 60))
    f %= PERIOD
    g, size = fof.fof_groups(f, PERIOD, S, nmin=25)
    for lab in np.unique(g[g >= 0]):
        members = np.nonzero(g == lab)[0]
        assert members.min() == lab and size[lab] == len(members) >= 25
    assert np.all(size[g < 0] < 25)


def cell_list_pairs(f, period, s_fixed, cell):
    # independent search: bin into cubic cells of side >= the linking length, compare 27 cells
    nc = period // cell
    c = f // cell
    key = (c[2] * nc + c[1]) * nc + c[0]
    buckets = {}
    for p, k in enumerate(key.tolist()):
        buckets.setdefault(k, []).append(p)
    pairs = set()
    for p in range(f.shape[1]):
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    k = (((c[2, p] + dz) % nc) * nc + (c[1, p] + dy) % nc) * nc + (c[0, p] + dx) % nc
                    for q in buckets.get(int(k), []):
                        if q <= p:
                            continue
                        d = (f[:, p] - f[:, q] + period // 2) % period - period // 2
                        if 25 * int(np.dot(d, d)) < s_fixed * s_fixed:
                            pairs.add((p, q))
    return pairs


def test_brute_force_pairs_equal_a_cell_list_search():
    rng = np.random.default_rng(5)
    centres = rng.integers(0, PERIOD, size=(3, 6))
    pick = rng.integers(0, 6, size=500)
    f = (centres[:, pick] + rng.normal(0, 40000, size=(3, 500)).astype(np.int64)) % PERIOD
    i, j = fof.friend_pairs(f, PERIOD, S)
    assert set(zip(i.tolist(), j.tolist())) == cell_list_pairs(f, PERIOD, S, cell=2**16)


def test_mass_function_counts_halos_above_thresholds():
    group = np.array([0, 0, 0, -1, 4, 4, -1])
    size = np.array([3, 3, 3, 1, 2, 2, 1])
    assert fof.mass_function(group, size, [1, 2, 3, 4]).tolist() == [2, 2, 1, 0]


def test_tree_candidates_give_the_brute_force_pairs():
    rng = np.random.default_rng(8)
    centres = rng.integers(0, PERIOD, size=(3, 10))
    pick = rng.integers(0, 10, size=3000)
    f = (centres[:, pick] + rng.normal(0, 60000, size=(3, 3000)).astype(np.int64)) % PERIOD
    f[:, :20] = np.array([[0], [5], [7]]) + np.arange(20) * 39321 * np.array([[1], [0], [0]])  # on the threshold
    f %= PERIOD
    for b in ((1, 5), (1, 4), (2, 7)):
        bi, bj = fof.friend_pairs(f, PERIOD, S, *b, method="brute")
        ti, tj = fof.friend_pairs(f, PERIOD, S, *b, method="tree")
        assert set(zip(bi.tolist(), bj.tolist())) == set(zip(ti.tolist(), tj.tolist()))
