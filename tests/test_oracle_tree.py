"""Pins for the quadtree, near lists and proxy circles."""
import numpy as np

from oracle import geometry, tree
from paper_2603_09381_gb300 import workloads as wl


def test_morton_order():
    assert [tree.morton(x, y) for x, y in [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0)]] == [0, 1, 2, 3, 4]


def test_circle_grid_near_lists_and_levels():
    prob = wl.circle_grid(4, 4, n=32)
    nds = geometry.all_nodes(prob)
    t = tree.build(prob, nds, {"tol": 1e-10})
    assert t["L"] == 2
    lv = t["levels"]
    assert [len(lv[l]) for l in (2, 1, 0)] == [16, 4, 1]
    keys = [b["key"] for b in lv[2]]
    assert keys[:4] == [(0, 0), (1, 0), (0, 1), (1, 1)]
    # leaf: r_cell = 0.4, R_p = 0.6; edge neighbours' nodes at 0.6 -> near by adjacency,
    # corner nodes at sqrt(2)-0.4 > 0.6 -> far
    for b in lv[2]:
        assert abs(b["r_cell"] - 0.4) < 1e-12
        nk = sorted(lv[2][o]["key"] for o in b["near"])
        x, y = b["key"]
        expect = sorted((x + dx, y + dy) for dx, dy in [(1, 0), (-1, 0), (0, 1), (0, -1)]
                        if 0 <= x + dx < 4 and 0 <= y + dy < 4)
        assert nk == expect
    # level 1: box of 2x2 circles, r_cell = sqrt(0.5) + 0.4, R_p = 1.5 r_cell = 1.6607;
    # the corner box's nearest nodes are at sqrt(2)*1.5 - 0.4 = 1.7213 > R_p -> far
    b = lv[1][0]
    assert abs(b["r_cell"] - (np.sqrt(0.5) + 0.4)) < 1e-12
    assert sorted(lv[1][o]["key"] for o in b["near"]) == [(0, 1), (1, 0)]


def test_proxy_circle_separates_far_nodes():
    prob = wl.star_grid(8, 8, n=64)
    nds = geometry.all_nodes(prob)
    t = tree.build(prob, nds, {"tol": 1e-10})
    for lev, boxes in t["levels"].items():
        for bi, b in enumerate(boxes):
            own = np.concatenate([nds[j]["x"] for j in b["leaves"]])
            assert np.max(np.hypot(*(own - b["center"]).T)) < b["R_p"]
            for bj, o in enumerate(boxes):
                if bj == bi or bj in b["near"]:
                    continue
                pts = np.concatenate([nds[j]["x"] for j in o["leaves"]])
                assert np.min(np.hypot(*(pts - b["center"]).T)) >= b["R_p"]


def test_padding_and_ragged_grid():
    prob = wl.circle_grid(3, 2, n=32)
    nds = geometry.all_nodes(prob)
    t = tree.build(prob, nds, {"tol": 1e-8})
    assert t["L"] == 2
    assert len(t["levels"][2]) == 6
    assert len(t["levels"][1]) == 2
    assert sorted(len(b["leaves"]) for b in t["levels"][1]) == [2, 4]


def test_arbitrary_arrangement_tree():
    """spacing 0: the bounding square of the centres at the smallest depth that
    gives every centre its own cell; leaves centred on their inclusions; every
    node of a non-near box outside the proxy circle at every level."""
    prob = wl.random_arrangement(20, seed=6)
    nds = geometry.all_nodes(prob)
    cent = np.array([[i["cx"], i["cy"]] for i in prob["inclusions"]])
    origin, cell, L, ij = tree.auto_cells(cent)
    assert len({tuple(x) for x in ij}) == 20 and ij.min() >= 0 and ij.max() < 2 ** L
    coarser = np.floor((cent - origin) / (2 * cell)).astype(int)
    assert len({tuple(x) for x in coarser}) < 20            # one level less would not separate them
    t = tree.build(prob, nds, {"tol": 1e-10})
    assert t["L"] == L
    for b in t["levels"][L]:
        assert np.allclose(b["center"], cent[b["leaves"][0]])
    for lev in range(1, L + 1):
        boxes = t["levels"][lev]
        for bi, b in enumerate(boxes):
            for bj, o in enumerate(boxes):
                if bj == bi or bj in b["near"]:
                    continue
                pts = np.concatenate([nds[j]["x"] for j in o["leaves"]])
                assert np.min(np.hypot(*(pts - b["center"]).T)) >= b["R_p"]
