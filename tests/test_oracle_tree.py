"""Pins of the oracle's octree and groups (Sect. 2, "construction of the
tree-datastructure"; groups per the vector-machine walk it cites).

Reference construction here: a recursive Python split of sorted keys into
octants, then a breadth-first numbering -- a different algorithm from the
oracle's level-by-level loop -- plus invariants any valid tree obeys."""
import numpy as np
import pytest

from paper_1204_2280_gb300 import workloads as W

L = 21


def digit(k, lev):
    return (int(k) >> (3 * (L - lev))) & 7


def brute_tree(skeys, nleaf):
    """Recursive octree; returns cells in BFS order as tuples
    (begin, count, level, nchild) with child lists."""
    n = len(skeys)
    nodes = []          # (begin, count, level, children)

    def rec(b, e, lev):
        me = {"b": b, "c": e - b, "l": lev, "ch": []}
        if e - b > nleaf and lev < L:
            s = b
            while s < e:
                d = digit(skeys[s], lev + 1)
                t = s
                while t < e and digit(skeys[t], lev + 1) == d:
                    t += 1
                me["ch"].append(rec(s, t, lev + 1))
                s = t
        return me

    root = rec(0, n, 0)
    # BFS numbering
    order = [root]
    i = 0
    while i < len(order):
        order.extend(order[i]["ch"])
        i += 1
    return order


def clustered_keys(rng, n):
    k = rng.integers(0, 1 << 63, n, dtype=np.uint64)
    k[: n // 4] = k[0] ^ rng.integers(0, 64, n // 4).astype(np.uint64)      # deep cluster
    k[n // 4: n // 4 + 40] = k[1]                                           # identical keys
    return np.sort(k)


@pytest.mark.parametrize("nleaf", [1, 4, 16])
@pytest.mark.parametrize("seed", [0, 1])
def test_tree_matches_recursive_construction(orc, nleaf, seed):
    sk = clustered_keys(np.random.default_rng(seed), 1500)
    t = orc.build_tree(sk, nleaf)
    ref = brute_tree(sk, nleaf)
    assert t.ncells == len(ref)
    idx = {id(c): i for i, c in enumerate(ref)}
    for i, c in enumerate(ref):
        assert t.body_begin[i] == c["b"] and t.body_count[i] == c["c"] and t.level[i] == c["l"]
        assert t.nchild[i] == len(c["ch"])
        if c["ch"]:
            assert t.child_begin[i] == idx[id(c["ch"][0])]
            assert [idx[id(x)] for x in c["ch"]] == list(range(t.child_begin[i], t.child_begin[i] + len(c["ch"])))


@pytest.mark.parametrize("n,nleaf", [(1, 16), (16, 16), (17, 16), (5000, 16), (5000, 8)])
def test_tree_invariants_plummer(orc, n, nleaf):
    b = W.plummer(n, 3)
    k = orc.keys(b.pos)
    sk = k[orc.sort(k)]
    t = orc.build_tree(sk, nleaf)
    leaf = t.nchild == 0
    # leaves partition the bodies
    assert t.body_count[leaf].sum() == n
    cover = np.zeros(n, int)
    for bb, cc in zip(t.body_begin[leaf], t.body_count[leaf]):
        cover[bb:bb + cc] += 1
    assert np.all(cover == 1)
    # leaf iff count <= nleaf or deepest level
    assert np.array_equal(leaf, (t.body_count <= nleaf) | (t.level == L))
    # children partition parents and sit one level deeper
    for c in np.nonzero(~leaf)[0]:
        ch = np.arange(t.child_begin[c], t.child_begin[c] + t.nchild[c])
        assert np.all(t.level[ch] == t.level[c] + 1)
        assert np.all(t.parent[ch] == c)
        assert t.body_begin[ch[0]] == t.body_begin[c]
        assert np.all(t.body_begin[ch[1:]] == t.body_begin[ch[:-1]] + t.body_count[ch[:-1]])
        assert t.body_count[ch].sum() == t.body_count[c]
    # BFS order: levels non-decreasing, key order inside a level
    assert np.all(np.diff(t.level) >= 0)
    for lev in np.unique(t.level):
        assert np.all(np.diff(t.body_begin[t.level == lev]) > 0)
    # every body of a cell shares the cell's key prefix
    for c in range(t.ncells):
        sh = np.uint64(3 * (L - t.level[c]))
        pre = sk[t.body_begin[c]: t.body_begin[c] + t.body_count[c]] >> sh
        assert np.all(pre == pre[0])


@pytest.mark.parametrize("ncrit", [1, 8, 32, 64])
def test_groups_definition(orc, ncrit):
    sk = clustered_keys(np.random.default_rng(7), 3000)
    t = orc.build_tree(sk, 16)
    gb, gc = orc.groups(t, ncrit)
    # brute force: cells with count <= ncrit whose parent has > ncrit, plus
    # oversize leaves cut in runs of ncrit
    want = []
    for c in range(t.ncells):
        if t.body_count[c] <= ncrit and (c == 0 or t.body_count[t.parent[c]] > ncrit):
            want.append((t.body_begin[c], t.body_count[c]))
        elif t.nchild[c] == 0 and t.body_count[c] > ncrit:
            for o in range(0, t.body_count[c], ncrit):
                want.append((t.body_begin[c] + o, min(ncrit, t.body_count[c] - o)))
    want.sort()
    assert list(zip(gb.tolist(), gc.tolist())) == [(int(a), int(b)) for a, b in want]
    # groups partition the bodies in key order
    assert gb[0] == 0 and np.all(gb[1:] == gb[:-1] + gc[:-1]) and gb[-1] + gc[-1] == 3000
    assert np.all(gc <= ncrit) and np.all(gc >= 1)


def _minimal_groups_brute(sk, nleaf, ncrit):
    """Groups of the unpacked rule from the recursive tree, as
    (begin, count, parent id or None) in key order."""
    out = []

    def rec(c, parent):
        if c["c"] <= ncrit and (parent is None or parent["c"] > ncrit):
            out.append((c["b"], c["c"], None if parent is None else id(parent)))
            return
        if not c["ch"] and c["c"] > ncrit:
            for o in range(0, c["c"], ncrit):
                out.append((c["b"] + o, min(ncrit, c["c"] - o), None))
            return
        for ch in c["ch"]:
            rec(ch, c)

    rec(brute_tree(sk, nleaf)[0], None)
    return out


@pytest.mark.parametrize("ncrit", [1, 8, 32, 64])
@pytest.mark.parametrize("seed", [7, 8])
def test_packed_groups_brute_force(orc, ncrit, seed):
    """Sibling packing: walking the recursive tree's unpacked groups in key
    order, a group joins the previous packed group when both come from the
    same parent cell and the sum stays <= ncrit."""
    sk = clustered_keys(np.random.default_rng(seed), 3000)
    t = orc.build_tree(sk, 16)
    gb, gc = orc.groups(t, ncrit, pack=True)
    want = []
    prev_parent = None
    for b, c, par in _minimal_groups_brute(sk, 16, ncrit):
        if want and par is not None and par == prev_parent and want[-1][1] + c <= ncrit:
            want[-1][1] += c
        else:
            want.append([b, c])
        prev_parent = par
    assert [[int(a), int(b)] for a, b in zip(gb, gc)] == want


@pytest.mark.parametrize("ncrit", [8, 32, 64])
def test_packed_groups_invariants_plummer(orc, ncrit):
    """Every packed group is a run of consecutive children of one cell, each
    child within ncrit bodies; the groups partition the bodies in key order;
    packing is greedy (a following sibling that would fit was not left out);
    and packing only merges unpacked groups."""
    n = 20000
    b = W.plummer(n, 5)
    k = orc.keys(b.pos)
    sk = k[orc.sort(k)]
    t = orc.build_tree(sk, 16)
    g0b, g0c = orc.groups(t, ncrit)
    gb, gc = orc.groups(t, ncrit, pack=True)
    assert gb[0] == 0 and np.all(gb[1:] == gb[:-1] + gc[:-1]) and gb[-1] + gc[-1] == n
    assert np.all(gc <= ncrit) and np.all(gc >= 1)
    assert set(gb.tolist()) <= set(g0b.tolist())          # boundaries are unpacked boundaries
    assert len(gb) < len(g0b)
    # cell lookup by (begin, count): the shallowest such cell (a cell with one
    # child has its child's range; BFS order lists the parent first)
    cell = {}
    for i, (bb, cc) in enumerate(zip(t.body_begin, t.body_count)):
        cell.setdefault((int(bb), int(cc)), i)
    par0 = np.array([t.parent[cell[(int(x), int(y))]] if (int(x), int(y)) in cell and cell[(int(x), int(y))] != 0
                     else -1 for x, y in zip(g0b, g0c)])
    start = {int(x): i for i, x in enumerate(g0b)}
    for j, (x, y) in enumerate(zip(gb, gc)):
        i0 = start[int(x)]
        i1 = i0
        while g0b[i1] + g0c[i1] < x + y:
            i1 += 1
        members = np.arange(i0, i1 + 1)
        assert g0c[members].sum() == y
        if len(members) > 1:                                # one parent, consecutive children
            p = par0[members[0]]
            assert p >= 0 and np.all(par0[members] == p)
            kids = [cell[(int(g0b[m]), int(g0c[m]))] for m in members]
            assert kids == list(range(kids[0], kids[0] + len(kids)))
        nxt = i1 + 1                                        # greedy: the next sibling did not fit
        if nxt < len(g0b) and par0[nxt] >= 0 and par0[nxt] == par0[i1]:
            assert y + g0c[nxt] > ncrit
