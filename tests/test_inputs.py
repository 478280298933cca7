"""Input generators: quadrature rule, meshes, list builders (exact cover)."""
import math

import numpy as np
import pytest

from tsqbx_inputs import configs, lists as L, mesh


def test_rule6_exact_to_degree_4():
    """The six-point rule integrates x^a y^b, a+b <= 4, exactly over the
    reference triangle (integral = a! b! / (a+b+2)!), and not degree 5."""
    bary, w = mesh.rule6_barycentric()
    # reference triangle (0,0), (1,0), (0,1), area 1/2
    P = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    xy = bary @ P
    for a in range(5):
        for b in range(5 - a):
            approx = 0.5 * np.sum(w * xy[:, 0] ** a * xy[:, 1] ** b)
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert approx == pytest.approx(exact, rel=1e-13, abs=1e-15)
    deg5 = [abs(0.5 * np.sum(w * xy[:, 0] ** a * xy[:, 1] ** (5 - a)) -
                math.factorial(a) * math.factorial(5 - a) / math.factorial(7)) for a in range(6)]
    assert max(deg5) > 1e-6
    assert np.all(bary > 0) and np.allclose(bary.sum(1), 1)


def test_meshes_counts_and_orientation():
    V, F = mesh.icosphere(3)
    assert F.shape == (1280, 3)
    F = mesh.orient_outward(V, F, lambda c: np.zeros_like(c))
    xyz, w, nrm, h, wex = mesh.nodes_on_triangles(V, F)
    assert xyz.shape == (7680, 3)
    assert np.all(np.einsum("ij,ij->i", nrm, xyz) > 0)           # outward
    assert w.sum() == pytest.approx(wex.sum(), rel=1e-12)
    assert w.sum() == pytest.approx(4 * np.pi, rel=0.01)           # inscribed sphere area
    V, F = mesh.torus(256, 96)
    assert F.shape == (49152, 3)
    V, F = mesh.geodesic_sphere(5)
    assert F.shape == (20 * 25, 3)


def test_lists_to_csr_roundtrip(rng):
    lists = [np.sort(rng.choice(100, size=rng.integers(0, 40), replace=False)) for _ in range(20)]
    grs, rb, re = L.lists_to_csr(lists)
    for i, x in enumerate(lists):
        got = np.concatenate([np.arange(rb[r], re[r]) for r in range(grs[i], grs[i + 1])] + [[]])
        np.testing.assert_array_equal(got.astype(int), x)
        # maximal runs: consecutive ranges of one group never touch
        for r in range(grs[i] + 1, grs[i + 1]):
            assert rb[r] > re[r - 1]


def test_sphere_workload_shape():
    g, mu = configs.sphere()
    assert (g.n_src, g.n_ctr, g.n_tgt, g.n_group) == (7680, 7680, 7680, 7680)
    per = g.group_source_counts()
    assert 100 < per.mean() < 400
    # every list is convergent: |t-c| < |s-c|
    import oracle
    nd, nz = oracle.count_divergent(g)
    assert nd == 0 and nz == 0


def _exact_cover_failures(tree):
    """For every target box b: List 1, List 3 close, List 4 close, List 3 far and
    the far field reached through List 2 / List 4 far of b and its ancestors
    (Alg. 1 Stages 3-8) must cover every source exactly once."""
    n = tree.n_src
    bad = []
    for b in np.nonzero(tree.n_owned_ctr > 0)[0]:
        d = np.zeros(n + 1, np.int64)
        boxes = []
        for nm in ("L1", "L3close", "L4close", "L3far"):
            boxes += list(tree.box_list(nm, b))
        for w in tree.ancestors(b):
            boxes += list(tree.box_list("L2", w)) + list(tree.box_list("L4far", w))
        for x in boxes:
            d[tree.src_begin[x]] += 1
            d[tree.src_end[x]] -= 1
        cnt = np.cumsum(d)[:n]
        if not np.all(cnt == 1):
            bad.append(int(b))
    return bad


@pytest.mark.parametrize("nu,nv,n_max", [(32, 12, 64), (40, 16, 16)])
def test_octree_exact_cover_torus(nu, nv, n_max):
    g, mu, tree = configs.torus(nu, nv, n_max=n_max)
    assert _exact_cover_failures(tree) == []
    # near lists are exactly List 1 + List 3 close + List 4 close
    assert g.n_pairs() > 0


def test_octree_exact_cover_cloud_with_nonleaf_owners(rng):
    """Random sources; big QBX balls stay in parent boxes (non-leaf target boxes)."""
    src = rng.uniform(-1, 1, (3000, 3))
    ctr = rng.uniform(-1, 1, (1500, 3))
    rad = np.where(rng.uniform(size=1500) < 0.3, 0.2, 0.01)
    tree = L.Octree(src, ctr, rad, n_max=20, t_f=0.9, n_mpole=10)
    nonleaf_targets = np.sum((tree.n_owned_ctr > 0) & (tree.is_leaf == 0))
    assert nonleaf_targets > 0
    assert _exact_cover_failures(tree) == []
    # every center is owned by a box whose TCR contains its ball
    for c in range(0, 1500, 37):
        b = tree.ctr_box[c]
        dist = np.linalg.norm(ctr[c] - tree.center[:, b])
        assert dist + rad[c] <= np.sqrt(3) * tree.halfwidth[b] * 1.9 + 1e-12 or b == 0


def test_octree_sources_sorted_by_box(rng):
    src = rng.uniform(-1, 1, (2000, 3))
    tree = L.Octree(src, src[:10] + 0.001, np.full(10, 1e-3), n_max=32)
    assert sorted(tree.src_perm.tolist()) == list(range(2000))
    sp = src[tree.src_perm]
    for b in range(tree.n_boxes):
        pts = sp[tree.src_begin[b]:tree.src_end[b]]
        if len(pts):
            assert np.all(np.abs(pts - tree.center[:, b]) <= tree.halfwidth[b] + 1e-12)


def test_near_targets_stay_convergent():
    """Extra targets per center lie within the original target's distance of
    their center, so every listed pair stays convergent."""
    import oracle
    from tsqbx_inputs import configs
    g, mu, _ = configs.torus_near_targets(24, 10, targets_per_center=5)
    assert g.n_tgt == 5 * g.n_ctr
    assert np.bincount(g.tgt_center, minlength=g.n_ctr).tolist() == [5] * g.n_ctr
    rho = np.linalg.norm(g.tgt_xyz - g.ctr_xyz[:, g.tgt_center], axis=0)
    assert np.all(rho[g.n_ctr:] <= rho[g.tgt_center[g.n_ctr:]] * (1 + 1e-12))
    nd, nz = oracle.count_divergent(g)
    assert nd == 0 and nz == 0


def test_near_targets_mixed_counts():
    """targets_per_center = "mixed:M": each center gets 1..M targets,
    log-uniformly (both sides of the conventional path's break-even), every
    extra target inside its center's convergence radius, seeded."""
    import oracle
    from tsqbx_inputs import configs
    g, mu, _ = configs.torus_near_targets(24, 10, targets_per_center="mixed:64")
    cnt = np.bincount(g.tgt_center, minlength=g.n_ctr)
    assert cnt.min() >= 1 and cnt.max() <= 64
    assert (cnt == 1).any() and (cnt >= 32).any()
    # log-uniform on [1, 64]: about half the centers have at most 8 targets
    assert 0.35 < np.mean(cnt <= 8) < 0.65
    rho = np.linalg.norm(g.tgt_xyz - g.ctr_xyz[:, g.tgt_center], axis=0)
    assert np.all(rho[g.n_ctr:] <= rho[g.tgt_center[g.n_ctr:]] * (1 + 1e-12))
    nd, nz = oracle.count_divergent(g)
    assert nd == 0 and nz == 0
    g2, _, _ = configs.torus_near_targets(24, 10, targets_per_center="mixed:64")
    assert np.array_equal(g.tgt_xyz, g2.tgt_xyz)


def _max_rho_over_R(g):
    """max over listed pairs of |t - c| / |s - c| (each center is its own
    group with one window of sources)."""
    C, S = g.ctr_xyz.T, g.src_xyz.T
    rho = np.linalg.norm(g.tgt_xyz.T - C[g.tgt_center], axis=1)
    L = (g.range_end - g.range_begin).astype(np.int64)
    mind = np.empty(len(C))
    for Lv in np.unique(L):
        idx = np.nonzero(L == Lv)[0]
        step = max(1, 2_000_000 // int(Lv))
        for a in range(0, len(idx), step):
            ii = idx[a:a + step]
            d = S[g.range_begin[ii][:, None] + np.arange(Lv)[None, :]] - C[ii][:, None, :]
            mind[ii] = np.sqrt(np.min(np.einsum("ijk,ijk->ij", d, d), axis=1))
    return float(np.max(rho / mind[g.tgt_center]))


def test_batched_surfaces_stay_well_inside_convergence():
    """The batched ellipsoids: the coarse, strongly curved ones (frequency
    <= 12, where a window of sources comes closest to a center relative to
    its target) keep every listed pair at rho/R <= 0.9.  Over the whole
    batch the maximum is 0.58."""
    from tsqbx_inputs import configs
    surfaces = configs.ellipsoid_batch()
    small = [g for g, _ in surfaces if g.n_src <= 120 * 12 ** 2]
    assert len(small) >= 10
    for g in small:
        assert _max_rho_over_R(g) <= 0.9, g.meta["name"]
