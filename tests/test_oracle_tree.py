"""Pins of the oracle's tree and interaction lists against what the paper and
plain counting fix (no GPU).

  - Fig. sdomain01: counter-clockwise box numbering at levels 1 and 2
  - Fig. hodlr2d_mat: the printed level-1 and level-2 block patterns
  - closed-form per-level counts of self / edge / vertex / far blocks on a
    full 2^l x 2^l grid of boxes (derived below, independent of the oracle)
  - exact once-coverage of every matrix entry
  - |E| <= 4, |I| <= 15 (attained), <= 5 dense blocks per leaf row (Sec. 4.1)
  - the leaf rule of Alg. 1 checked by an independent histogram
"""
import os

import numpy as np
import pytest

from paper_2204_05536_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig_hodlr2d_mat.txt")


def _grid_points(level, per_cell=1, seed=0):
    """per_cell points strictly inside every cell of a 2^level grid on [0,1]^2."""
    m = 2 ** level
    rng = np.random.default_rng(seed)
    pts = []
    for iy in range(m):
        for ix in range(m):
            for _ in range(per_cell):
                pts.append(((ix + rng.uniform(0.2, 0.8)) / m, (iy + rng.uniform(0.2, 0.8)) / m))
    return np.array(pts)


def _read_golden():
    pats, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("level"):
            cur = int(line.split()[1])
            pats[cur] = []
        else:
            pats[cur].append(line)
    return pats


def test_numbering_matches_fig_sdomain01(oracle):
    # level 1: 0 bottom-left, 1 bottom-right, 2 top-right, 3 top-left
    assert [oracle.paper_coords(1, b) for b in range(4)] == [(0, 0), (1, 0), (1, 1), (0, 1)]
    # level 2, read off the figure: box -> (column, row) from the bottom-left
    fig = {0: (0, 0), 1: (1, 0), 3: (0, 1), 2: (1, 1), 4: (2, 0), 5: (3, 0), 7: (2, 1),
           6: (3, 1), 12: (0, 2), 13: (1, 2), 15: (0, 3), 14: (1, 3), 8: (2, 2), 9: (3, 2),
           11: (2, 3), 10: (3, 3)}
    for b, xy in fig.items():
        assert oracle.paper_coords(2, b) == xy
        assert oracle.paper_index(2, *xy) == b


def test_paper_numbering_roundtrip(oracle):
    for level in range(5):
        seen = set()
        for b in range(4 ** level):
            ix, iy = oracle.paper_coords(level, b)
            assert oracle.paper_index(level, ix, iy) == b
            seen.add((ix, iy))
        assert len(seen) == 4 ** level
        # children of b are 4b..4b+3 and lie inside b
        if level >= 1:
            for b in range(4 ** (level - 1)):
                px, py = oracle.paper_coords(level - 1, b)
                for c in range(4):
                    cx, cy = oracle.paper_coords(level, 4 * b + c)
                    assert (cx >> 1, cy >> 1) == (px, py)


@pytest.mark.parametrize("level", [1, 2])
def test_block_pattern_matches_fig_hodlr2d_mat(oracle, level):
    pts = _grid_points(level, per_cell=2)
    k = oracle.kernel("imq", a=0.01)
    o = oracle.Oracle(pts, k, leaf_size=1000, eps=1e-8, root=(0.0, 0.0, 1.0), levels=level,
                      compress=False)
    want = _read_golden()[level]
    nb = 4 ** level
    for a in range(nb):
        row = []
        for b in range(nb):
            if a == b:
                ch = "S"
            elif b in o.edge_list(level, a):
                ch = "E"
            elif b in o.interaction_list(level, a):
                ch = "L"
            elif level == 2 and (b // 4) in o.interaction_list(1, a // 4):
                ch = "1"
            else:
                ch = "?"
            row.append(ch)
        assert "".join(row) == want[a], "row %d" % a


def _closed_form_counts(level):
    """Ordered-pair counts on a full m x m grid, m = 2^l.
    edge:   horizontally or vertically adjacent cells, m(m-1) per direction,
            2 directions, 2 orders -> 4 m (m-1).
    vertex: diagonal neighbours, 4 (m-1)^2 ordered pairs, less those whose
            parents are themselves diagonal neighbours (for each such parent
            pair exactly one child pair meets at the shared corner):
            4 (m-1)^2 - 4 (m/2-1)^2.
    I:      every cell of the parent and of the parent's edge neighbours' 4
            children, minus self and own edge sharers:
            sum_C 4 (1 + |E(parent)|) - 1 - |E(C)| = 3 * 4^l + 16 E_{l-1} - E_l.
    far = I - vertex."""
    m = 2 ** level

    def edges(mm):
        return 4 * mm * (mm - 1)

    e = edges(m)
    if level == 0:
        return {"self": 1, "edge": 0, "vertex": 0, "far": 0}
    v = 4 * (m - 1) ** 2 - 4 * (m // 2 - 1) ** 2
    i_total = 3 * 4 ** level + 16 * edges(m // 2) - e
    return {"self": m * m, "edge": e, "vertex": v, "far": i_total - v}


def test_closed_form_counts_full_grid(oracle):
    L = 5
    pts = _grid_points(L)
    o = oracle.Oracle(pts, oracle.kernel("imq", a=0.01), leaf_size=1, eps=1e-8,
                      root=(0.0, 0.0, 1.0), compress=False)
    assert o.kappa == L
    # the paper's figure: level 1 has 4 self, 8 edge, 4 low-rank blocks;
    # level 2 has 16 self, 48 edge and 128 low-rank blocks
    assert _closed_form_counts(1) == {"self": 4, "edge": 8, "vertex": 4, "far": 0}
    c2 = _closed_form_counts(2)
    assert (c2["self"], c2["edge"], c2["vertex"] + c2["far"]) == (16, 48, 128)
    for level in range(L + 1):
        assert o.level_counts(level) == _closed_form_counts(level), level


def test_list_sizes_and_max_15(oracle):
    L = 4
    o = oracle.Oracle(_grid_points(L), oracle.kernel("imq", a=0.01), leaf_size=1, eps=1e-8,
                      root=(0.0, 0.0, 1.0), compress=False)
    for level in range(1, L + 1):
        sizes = [len(o.interaction_list(level, b)) for b in range(4 ** level)]
        esz = [len(o.edge_list(level, b)) for b in range(4 ** level)]
        assert max(esz) <= 4
        assert max(sizes) <= 15
        if level >= 3:
            assert max(sizes) == 15  # interior boxes reach the bound of Sec. 4.1
        assert max(1 + e for e in esz) <= 5  # dense blocks per leaf row


@pytest.mark.parametrize("dist", ["uniform", "clustered"])
def test_exact_once_coverage(oracle, dist):
    rng = np.random.default_rng(3)
    if dist == "uniform":
        pts = inputs.uniform(600, seed=5)
    else:  # two tight clusters plus a sparse background -> many empty boxes
        pts = np.concatenate([rng.normal(0.5, 0.02, (250, 2)), rng.normal(-0.6, 0.05, (250, 2)),
                              rng.uniform(-1, 1, (100, 2))])
    o = oracle.Oracle(pts, oracle.kernel("imq", a=0.01), leaf_size=8, eps=1e-8, compress=False)
    assert o.kappa >= 3
    mark = o.coverage()
    assert mark.min() == 1 and mark.max() == 1


def test_leaf_rule_and_box_order(oracle):
    pts = inputs.uniform(3000, seed=0)
    nmax = 40
    o = oracle.Oracle(pts, oracle.kernel("imq", a=0.01), leaf_size=nmax, eps=1e-8,
                      root=(-1.0, -1.0, 2.0), compress=False)

    def max_count(level):
        m = 2 ** level
        ix = np.clip(np.floor((pts[:, 0] + 1.0) / 2.0 * m), 0, m - 1)
        iy = np.clip(np.floor((pts[:, 1] + 1.0) / 2.0 * m), 0, m - 1)
        _, c = np.unique(ix * m + iy, return_counts=True)
        return c.max()

    k = o.kappa
    assert max_count(k) <= nmax and max_count(k - 1) > nmax
    counts = o.box_counts(k)
    assert counts.sum() == len(pts)
    for b in range(0, 4 ** k, 37):
        p = o.box_points(k, b)
        assert np.all(np.diff(p) > 0)  # ascending original index
        ix, iy = oracle.paper_coords(k, b)
        m = 2 ** k
        lo = np.array([ix, iy]) / m * 2.0 - 1.0
        assert np.all(pts[p] >= lo - 1e-15) and np.all(pts[p] <= lo + 2.0 / m + 1e-15)


def test_boundary_points_clamp(oracle):
    # points on the outer max edge go to the last box; interior edges go right/up
    pts = np.array([[1.0, 1.0], [0.0, 0.0], [-1.0, -1.0], [0.5, -1.0], [1.0, 0.25]])
    o = oracle.Oracle(pts, oracle.kernel("imq", a=0.1), leaf_size=1, eps=1e-8,
                      root=(-1.0, -1.0, 2.0), levels=2, compress=False)
    where = {}
    for b in range(16):
        for p in o.box_points(2, b):
            where[int(p)] = oracle.paper_coords(2, b)
    assert where[0] == (3, 3) and where[1] == (2, 2) and where[2] == (0, 0)
    assert where[3] == (3, 0) and where[4] == (3, 2)
