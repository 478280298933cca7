"""The host octree builder against the interaction-list definitions of Sec. 3.2
(Defs. 1-9), evaluated by brute force over every pair of boxes.

The builder finds its lists by tree walks (adjacent leaves from the root, List 3
below the 2-colleagues' children, List 4 by a descent over coarser boxes, the
close/far split by recursive classification).  Here every list is the set that
its definition names, formed by testing each box of the tree against each
other one, so that a walk that prunes too early or too late, a wrong level
test or a wrong separation constant shows up as a set difference.  The exact
cover test (tests/test_inputs.py) adds that the lists partition the sources.

Readings (as in the builder): boxes are adjacent when the closed boxes
intersect; a < TCR(b) means the center of a is outside TCR(b) by at least 3|a|;
TCR(a) < b uses the l-infinity distance (Sec. 3.1).  Empty boxes carry no
interactions and are left out of every list.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from tsqbx_inputs import configs
from tsqbx_inputs import lists as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class Boxes:
    """Box geometry and the relations of Sec. 3.1 as dense boolean matrices."""

    def __init__(self, tree):
        self.t = tree
        nb = self.nb = tree.n_boxes
        self.C = tree.center.T.copy()
        self.H = tree.halfwidth.copy()
        self.lev = tree.level.astype(np.int64)
        self.par = tree.parent.astype(np.int64)
        self.leaf = tree.is_leaf.astype(bool)
        self.ns = (tree.src_end - tree.src_begin).astype(np.int64)
        self.target = tree.n_owned_ctr > 0
        # anc[d, a]: a is a strict ancestor of d
        self.anc = np.zeros((nb, nb), bool)
        for d in range(nb):
            a = self.par[d]
            while a >= 0:
                self.anc[d, a] = True
                a = self.par[a]
        self.target_or_anc = self.target | self.anc[self.target].any(axis=0)
        D = np.abs(self.C[:, None, :] - self.C[None, :, :])            # |c_a - c_b| per axis
        # closed boxes intersect (their boundaries meet, or one holds the other)
        self.adj = np.all(D <= self.H[:, None, None] + self.H[None, :, None], axis=2)
        # d is a 2-colleague of b: same level, inside the box of radius |b|(1 + 2*2) about c_b
        same = self.lev[:, None] == self.lev[None, :]
        self.coll2 = same & np.all(D + self.H[:, None, None] <= 5.0 * self.H[None, :, None], axis=2)
        # a < TCR(b): |c_a - c_b| - sqrt(3)|b|(1 + t_f) >= 3|a|
        d2 = np.zeros((nb, nb))
        for k in range(3):
            d2 = d2 + (self.C[:, None, k] - self.C[None, :, k]) * (self.C[:, None, k] - self.C[None, :, k])
        tcr = np.sqrt(3.0) * self.H * (1.0 + tree.t_f)
        self.sep_box_tcr = np.sqrt(d2) - tcr[None, :] >= 3.0 * self.H[:, None]
        # TCR(a) < d: l-infinity distance from c_a to box d >= 3|a|(1 + t_f)
        linf = np.maximum(0.0, (D - self.H[None, :, None]).max(axis=2))
        self.sep_tcr_box = linf >= 3.0 * self.H[:, None] * (1.0 + tree.t_f)

    def source_leaf(self):
        return self.leaf & (self.ns > 0)


def definition_lists(B):
    """Every list of Sec. 3.2 for every box it is defined on, from Defs. 1-9."""
    nb, t = B.nb, B.t
    out = {k: [set() for _ in range(nb)] for k in ("L1", "L2", "L3", "L4", "L3far", "L3close",
                                                     "L4close", "L4far")}
    boxes = np.arange(nb)
    srcleaf = B.source_leaf()
    for b in np.nonzero(B.target_or_anc)[0]:
        # Def. 3 (List 2): children of the 2-colleagues of parent(b), 2-well-separated from b
        if B.par[b] >= 0:
            pc = B.coll2[:, B.par[b]]
            sel = (B.par >= 0) & pc[np.maximum(B.par, 0)] & (B.lev == B.lev[b]) & ~B.coll2[:, b] & (B.ns > 0)
            out["L2"][b] = set(boxes[sel].tolist())
        # Def. 5 (List 4): source boxes that are 2-colleagues of an ancestor of b,
        # adjacent to parent(b) and not to b; and 2-colleagues of b not adjacent to b
        sel = srcleaf & B.coll2[:, b] & ~B.adj[:, b]
        if B.par[b] >= 0:
            anc_b = np.nonzero(B.anc[b])[0]
            coll_anc = B.coll2[:, anc_b].any(axis=1)
            sel |= srcleaf & coll_anc & B.adj[:, B.par[b]] & ~B.adj[:, b]
        out["L4"][b] = set(boxes[sel].tolist())
    for b in np.nonzero(B.target_or_anc)[0]:
        chain = [b] + np.nonzero(B.anc[b])[0].tolist()
        # Def. 8 (List 4 close): in List 4 of b or an ancestor, TCR(b) not < d
        l4c = set()
        for w in chain:
            l4c |= {d for d in out["L4"][w] if not B.sep_tcr_box[b, d]}
        out["L4close"][b] = l4c
    for b in np.nonzero(B.target_or_anc)[0]:
        # Def. 9 (List 4 far)
        l4f = {d for d in out["L4"][b] if B.sep_tcr_box[b, d]}
        if B.par[b] >= 0:
            l4f |= {d for d in out["L4close"][B.par[b]] if B.sep_tcr_box[b, d]}
        out["L4far"][b] = l4f
    for b in np.nonzero(B.target)[0]:
        # Def. 2 (List 1): leaves among b, its descendants and the boxes adjacent to b
        sel = srcleaf & ((boxes == b) | B.anc[:, b] | B.adj[:, b])
        out["L1"][b] = set(boxes[sel].tolist())
        # Def. 4 (List 3): d strictly below some 2-colleague of b, not adjacent to
        # b, with every ancestor of d below the 2-colleagues adjacent to b
        Tb = np.nonzero(B.coll2[:, b])[0]
        below = B.anc[:, Tb].any(axis=1)                      # descendants(T_b)
        l3 = set()
        for d in np.nonzero(below & (B.ns > 0) & ~B.adj[:, b])[0]:
            ws = np.nonzero(B.anc[d] & below)[0]
            if np.all(B.adj[ws, b]):
                l3.add(int(d))
        out["L3"][b] = l3
        # the List 3 subtrees: List 3 boxes and their descendants
        l3arr = np.array(sorted(l3), dtype=np.int64)
        in3 = np.zeros(nb, bool)
        if len(l3arr):
            in3 = np.isin(boxes, l3arr) | B.anc[:, l3arr].any(axis=1)
        # far candidates: separated from TCR(b), no separated ancestor inside the subtrees
        cand = set()
        for d in np.nonzero(in3 & (B.ns > 0) & B.sep_box_tcr[:, b])[0]:
            ws = np.nonzero(B.anc[d] & in3)[0]
            if not np.any(B.sep_box_tcr[ws, b]):
                cand.add(int(d))
        # Def. 7 (List 3 far) and Def. 6 (List 3 close, leaves)
        out["L3far"][b] = {d for d in cand if B.ns[d] >= t.n_mpole}
        small = [d for d in cand if B.ns[d] < t.n_mpole]
        l3c = set()
        for d in np.nonzero(in3 & srcleaf)[0]:
            if not B.sep_box_tcr[d, b]:
                l3c.add(int(d))
            elif any(w == d or B.anc[d, w] for w in small):
                l3c.add(int(d))
        out["L3close"][b] = l3c
    return out


def leaves_under(B, boxes):
    """The nonempty leaves of the given boxes' subtrees."""
    res = set()
    for x in boxes:
        sel = B.source_leaf() & ((np.arange(B.nb) == x) | B.anc[:, x])
        res |= set(np.nonzero(sel)[0].tolist())
    return res


def compare(tree):
    """Set differences between the builder's lists and the definitions (empty
    when they agree), and a check of the merged near-field ranges."""
    B = Boxes(tree)
    ref = definition_lists(B)
    bad = []
    for name in ("L1", "L2", "L3", "L4", "L3far", "L4close", "L4far", "L3close"):
        for b in range(B.nb):
            got = tree.box_list(name, b).tolist()
            if name != "L3close" and len(set(got)) != len(got):
                bad.append((name, b, "duplicate"))
            gs = leaves_under(B, got) if name == "L3close" else set(got)
            if gs != ref[name][b]:
                bad.append((name, b, sorted(gs ^ ref[name][b])))
    # near ranges: the sources of List 1, List 3 close and List 4 close, merged
    for b in np.nonzero(B.target)[0]:
        cover = np.zeros(tree.n_src, np.int64)
        for x in ref["L1"][b] | ref["L3close"][b] | ref["L4close"][b]:
            cover[tree.src_begin[x]:tree.src_end[x]] += 1
        rb = tree.near_begin[tree.near_start[b]:tree.near_start[b + 1]]
        re = tree.near_end[tree.near_start[b]:tree.near_start[b + 1]]
        got = np.zeros(tree.n_src, np.int64)
        for x, y in zip(rb, re):
            got[x:y] += 1
        merged = np.all(rb[1:] > re[:-1]) and np.all(re > rb)
        if not (np.array_equal(cover, got) and merged and cover.max(initial=0) <= 1):
            bad.append(("near", int(b), "ranges"))
    return bad


def _trees():
    rng = np.random.default_rng(20191114)
    src = rng.uniform(-1, 1, (1500, 3))
    ctr = rng.uniform(-1, 1, (700, 3))
    rad = np.where(rng.uniform(size=700) < 0.3, 0.25, 0.02)
    yield "cloud, large balls", dict(src=src, ctr=ctr, rad=rad, n_max=20, t_f=0.9, n_mpole=10)
    # clustered sources: a deep, unbalanced tree, with coarse leaves beside fine ones
    c = rng.normal(0, 0.05, (1200, 3)) + np.array([0.4, -0.3, 0.2])
    src2 = np.concatenate([c, rng.uniform(-1, 1, (300, 3))])
    ctr2 = src2[::3] + rng.normal(0, 0.01, (len(src2[::3]), 3))
    rad2 = np.full(len(ctr2), 0.005)
    yield "clustered", dict(src=src2, ctr=ctr2, rad=rad2, n_max=12, t_f=0.5, n_mpole=30)
    yield "no confinement, no threshold", dict(src=src, ctr=ctr, rad=rad * 0.2, n_max=16, t_f=0.0, n_mpole=0)
    # the multipole threshold equal to a far candidate's source count (the
    # candidates do not depend on n_mpole; with n_mpole = 0 all are List 3 far)
    probe = L.Octree(src, ctr, rad, n_max=20, t_f=0.9, n_mpole=0)
    far = probe.lists["L3far"][1]
    counts = np.sort((probe.src_end - probe.src_begin)[far])
    yield "cloud, threshold at a candidate's count", dict(src=src, ctr=ctr, rad=rad, n_max=20, t_f=0.9,
                                                          n_mpole=int(counts[len(counts) // 2]))
    src3, ctr3, rad3 = configs.torus_points(24, 8)
    yield "torus 24x8", dict(src=src3, ctr=ctr3, rad=rad3, n_max=24, t_f=0.9, n_mpole=40)


TREE_NAMES = ["cloud, large balls", "clustered", "no confinement, no threshold",
              "cloud, threshold at a candidate's count", "torus 24x8"]
_TREES = None


def trees():
    """The cases, built on first use (not at collection)."""
    global _TREES
    if _TREES is None:
        _TREES = list(_trees())
        assert [n for n, _ in _TREES] == TREE_NAMES
    return _TREES


def _build(case, lib_path=None):
    return L.Octree(case["src"], case["ctr"], case["rad"], n_max=case["n_max"], t_f=case["t_f"],
                    n_mpole=case["n_mpole"], lib_path=lib_path)


@pytest.mark.parametrize("name", TREE_NAMES)
def test_builder_matches_definitions(name):
    case = dict(trees())[name]
    tree = _build(case)
    B = Boxes(tree)
    # the cases reach every list: non-leaf target boxes, List 3 far and close,
    # List 4 close and far (summed over the cases below)
    assert B.nb > 50
    assert compare(tree) == []


def test_cases_exercise_every_list():
    seen = {k: 0 for k in ("L2", "L3far", "L3close", "L4close", "L4far")}
    nonleaf_targets = 0
    for _, case in trees():
        tree = _build(case)
        for k in seen:
            seen[k] += len(tree.lists[k][1])
        nonleaf_targets += int(np.sum((tree.n_owned_ctr > 0) & (tree.is_leaf == 0)))
    assert all(v > 0 for v in seen.values()), seen
    assert nonleaf_targets > 0


# Plausible mistakes in the builder's walks and tests; each must change some
# list against its definition on one of the trees above.
BUILDER_MUTATIONS = {
    "adjacent_strict": ("> a.h + b.h) return false;", ">= a.h + b.h) return false;"),
    "colleague_one_away": ("> 4.0 * b.h) return false;", "> 2.0 * b.h) return false;"),
    "tcr_no_confinement": ("b.h * (1.0 + T.t_f); }", "b.h; }"),
    "sep_box_constant": (">= 3.0 * a.h;\n}", ">= 2.0 * a.h;\n}"),
    "sep_tcr_constant": ("return dist >= 3.0 * a.h * (1.0 + T.t_f);", "return dist >= 3.0 * a.h;"),
    "list4_level": ("if (x.level >= w.level || !adjacent(x, pw)) return;",
                    "if (x.level > w.level || !adjacent(x, pw)) return;"),
    "list3_stop": ("if (!adjacent(d, b)) { out.push_back(node); return; }",
                   "if (!adjacent(d, b)) { out.push_back(node); }"),
    "mpole_threshold": ("if (nsrc(w) >= T.n_mpole) far.push_back(node);",
                        "if (nsrc(w) > T.n_mpole) far.push_back(node);"),
    "list4far_parent": ("for (int d : T.lists[L4CLOSE][w.parent])",
                        "for (int d : T.lists[L4RAW][w.parent])"),
}


@pytest.mark.parametrize("name", sorted(BUILDER_MUTATIONS))
def test_definitions_catch_planted_builder_mistake(scratch, name):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    old, new = BUILDER_MUTATIONS[name]
    src = open(os.path.join(ROOT, "tsqbx_inputs", "octree.cpp")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mut = scratch / "octree_mut.cpp"
    mut.write_text(src.replace(old, new))
    lib = scratch / "liboctree_mut.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", str(mut),
                    "-o", str(lib)], check=True, capture_output=True)
    caught = False
    for _, case in trees():
        try:
            tree = _build(case, lib_path=str(lib))
        except ValueError:
            caught = True
            break
        if compare(tree):
            caught = True
            break
    assert caught, f"the definitions did not catch mutation {name}"
