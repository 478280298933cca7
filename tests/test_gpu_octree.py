"""GPU octree and near-field lists (tsqbx_octree_build) against the host
builder of the input tooling, which follows the same definitions (Sec.
3.1-3.2) and is pinned by the exact-cover tests in test_inputs.py.  Integer
and index results must agree exactly: box numbering and geometry, source
order, center ownership and every merged near-field range."""
import numpy as np
import pytest

from tsqbx_inputs import configs, lists as L, mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01110_gb300 as pkg
    pkg.lib()
    return pkg


def torus_points(nu, nv):
    V, F = mesh.torus(nu, nv, 1.0, 0.35)
    F = mesh.orient_outward(V, F, configs._torus_core)
    xyz, w, nrm, h = configs._surface_nodes(V, F)
    one = np.ones(len(xyz))
    C, Rr, T, Tn, node = mesh.centers_and_targets(xyz, nrm, h, [one, -one])
    return xyz, C, Rr


def compare(pkg, src, ctr, rad, **kw):
    ref = L.Octree(src, ctr, rad, **kw)
    got = pkg.Octree(src, ctr, rad, **kw)
    assert got.n_boxes == ref.n_boxes
    for name in ("level", "parent", "is_leaf", "n_owned_ctr", "src_begin", "src_end", "halfwidth",
                 "src_perm", "ctr_box", "near_start", "near_begin", "near_end"):
        a, b = getattr(got, name), getattr(ref, name)
        assert np.array_equal(np.asarray(a), np.asarray(b)), name
    assert np.array_equal(got.center, ref.center)
    return got, ref


@pytest.mark.parametrize("nu,nv", [(24, 10), (48, 18), (96, 36)])
def test_torus(pkg, nu, nv):
    src, ctr, rad = torus_points(nu, nv)
    got, _ = compare(pkg, src, ctr, rad)
    assert got.stats["n_target_boxes"] > 0 and got.stats["near_nnz"] > 0


@pytest.mark.parametrize("n_max,t_f,n_mpole", [(1, 0.9, 40), (4, 0.0, 0), (16, 1.5, 5), (64, 0.9, 40),
                                               (200, 0.9, 1000)])
def test_random_clouds(pkg, n_max, t_f, n_mpole):
    rng = np.random.default_rng(n_max * 7 + n_mpole)
    src = rng.uniform(-1, 1, (3000, 3))
    ctr = rng.uniform(-1, 1, (1500, 3))
    rad = rng.uniform(0.0, 0.05, 1500)
    compare(pkg, src, ctr, rad, n_max=n_max, t_f=t_f, n_mpole=n_mpole)


def test_clustered_deep_tree(pkg):
    """Points concentrated near a corner: a deep, unbalanced tree."""
    rng = np.random.default_rng(5)
    src = 0.25 + rng.exponential(1e-3, (4000, 3))
    src = np.concatenate([src, rng.uniform(-1, 1, (500, 3))])
    ctr = src[::7] + rng.normal(0, 1e-5, (len(src[::7]), 3))
    rad = np.full(len(ctr), 1e-5)
    got, _ = compare(pkg, src, ctr, rad, n_max=8)
    assert got.stats["max_level"] >= 8


def test_big_balls_stay_high(pkg):
    """Centers whose balls fit no child stay in upper boxes."""
    rng = np.random.default_rng(6)
    src = rng.uniform(-1, 1, (2000, 3))
    ctr = rng.uniform(-0.5, 0.5, (300, 3))
    rad = rng.uniform(0.3, 1.5, 300)
    got, _ = compare(pkg, src, ctr, rad, n_max=16)
    assert np.any(got.is_leaf[got.ctr_box] == 0)          # some centers own non-leaf boxes


def test_degenerate_inputs(pkg):
    rng = np.random.default_rng(7)
    src = rng.uniform(-1, 1, (100, 3))
    ctr = rng.uniform(-1, 1, (40, 3))
    rad = np.full(40, 0.01)
    compare(pkg, src, np.zeros((0, 3)), np.zeros(0))          # no centers
    compare(pkg, np.zeros((0, 3)), ctr, rad)                   # no sources
    compare(pkg, src[:1], ctr[:1], rad[:1])                    # one of each
    compare(pkg, src, ctr, rad, n_max=1000)                    # a single leaf


def test_lists_drive_the_same_pairs(pkg):
    """octree_lists from the GPU equals the host packaging used to build the
    benchmark geometries."""
    src, ctr, rad = torus_points(48, 18)
    g_tree, *g = pkg.octree_lists(src, ctr, rad)
    h_tree, *h = L.octree_lists(src, ctr, rad)
    for a, b in zip(g, h):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_rejects_overdeep_trees(pkg):
    src = np.zeros((100, 3))                                   # coincident sources
    with pytest.raises(pkg.TsqbxError) as ei:
        pkg.Octree(src, np.zeros((0, 3)), np.zeros(0), n_max=4)
    assert ei.value.code == -10
