"""The synthetic workloads (seeded).  Base seed 20191114; config i uses seed+i.

  sphere      -- Laplace SLP p=5: icosphere (3 subdivisions, 1280 flat triangles),
                 6 nodes per triangle, one center per node (alternating sides),
                 radius lists of 4h.
  torus       -- Laplace SLP+DLP p=9: torus R=1, r=0.35, 256 x 96 quads
                 (49,152 triangles, 294,912 sources), 2 centers per node,
                 GIGAQBX octree lists with n_max=64, t_f=0.9, n_mpole=40.
  torus_helm  -- Helmholtz SLP k=10 p=12: 444 x 166 quads (147,408 triangles,
                 884,448 sources), octree lists as above, plane-wave density.
  ellipsoids  -- 64 ellipsoids (semi-axes U(0.5,2)), log-uniform sizes, nearest
                 lists of log-uniform length 50..800, p in {5,7,9}.
  torus_near_targets -- the torus recipe with many targets per center (the
                 regime where conventional QBX is cheaper).
  urchin_points -- list-building inputs on the urchin surfaces gamma_k of
                 Sec. 5.1 as flat triangles.
Scaled-down variants (same recipe, fewer quads) serve the parity tests.
"""
import numpy as np

from . import density as dens
from . import lists as L
from . import mesh
from .geometry import Geometry

BASE_SEED = 20191114


def _surface_nodes(V, F, order_sources=True):
    xyz, w, nrm, h, wex = mesh.nodes_on_triangles(V, F)
    if order_sources:
        perm = mesh.morton_order(xyz)
        xyz, w, nrm, h, wex = xyz[perm], w[perm], nrm[perm], h[perm], wex[perm]
    return xyz, w, nrm, h


def _geometry_radius(xyz, w, nrm, h, signs, radius_factor):
    C, Rr, T, Tn, node = mesh.centers_and_targets(xyz, nrm, h, signs)
    grs, rb, re = L.radius_lists(xyz, C, radius_factor * h[node])
    n = len(C)
    return Geometry(np.ascontiguousarray(xyz.T), w, np.ascontiguousarray(nrm.T),
                    np.ascontiguousarray(C.T), Rr, np.ascontiguousarray(T.T),
                    np.arange(n, dtype=np.int32), np.ascontiguousarray(Tn.T),
                    np.arange(n, dtype=np.int32), grs, rb, re)


def _geometry_octree(xyz, w, nrm, h, signs, n_max=64, t_f=0.9, n_mpole=40):
    C, Rr, T, Tn, node = mesh.centers_and_targets(xyz, nrm, h, signs)
    tree, sperm, corder, cgroup, grs, rb, re = L.octree_lists(xyz, C, Rr, n_max, t_f, n_mpole)
    xyz, w, nrm = xyz[sperm], w[sperm], nrm[sperm]
    C, Rr, T, Tn = C[corder], Rr[corder], T[corder], Tn[corder]
    n = len(C)
    g = Geometry(np.ascontiguousarray(xyz.T), w, np.ascontiguousarray(nrm.T),
                 np.ascontiguousarray(C.T), Rr, np.ascontiguousarray(T.T),
                 np.arange(n, dtype=np.int32), np.ascontiguousarray(Tn.T),
                 cgroup, grs, rb, re)
    g.meta.update(n_boxes=int(tree.n_boxes), n_leaves=int(tree.is_leaf.sum()),
                  max_level=int(tree.level.max()), n_max=n_max, t_f=t_f, n_mpole=n_mpole)
    return g, tree


def sphere(seed_offset=0, subdiv=3):
    """Laplace SLP workload on the icosphere (radius lists of 4h)."""
    rng = np.random.default_rng(BASE_SEED + 0 + seed_offset)
    V, F = mesh.icosphere(subdiv)
    F = mesh.orient_outward(V, F, lambda c: np.zeros_like(c))
    xyz, w, nrm, h = _surface_nodes(V, F)
    sign = np.where(np.arange(len(xyz)) % 2 == 0, 1.0, -1.0)
    g = _geometry_radius(xyz, w, nrm, h, [sign], 4.0)
    g.meta.update(name=f"sphere-ico{subdiv}", kernel="laplace", p=5)
    return g, dens.sphere_density(xyz, rng)


def torus(nu=256, nv=96, seed_offset=0, n_max=64):
    """Laplace SLP+DLP workload on the torus with octree lists."""
    rng = np.random.default_rng(BASE_SEED + 1 + seed_offset)
    V, F = mesh.torus(nu, nv, 1.0, 0.35)
    F = mesh.orient_outward(V, F, _torus_core)
    xyz, w, nrm, h = _surface_nodes(V, F)
    one = np.ones(len(xyz))
    g, tree = _geometry_octree(xyz, w, nrm, h, [one, -one], n_max=n_max)
    g.meta.update(name=f"torus-{nu}x{nv}", kernel="laplace", p=9)
    src = g.src_xyz.T
    return g, dens.harmonic_density(src, rng), tree


def torus_near_targets(nu=96, nv=36, targets_per_center=16, seed_offset=0, n_max=64):
    """The torus recipe with many targets per QBX center (off-surface
    evaluation near the surface): besides its own target at half the ball
    radius, each center gets targets_per_center - 1 more, uniform in the ball
    of that same radius about the center (so |t-c| is never larger than for
    the original target and every pair stays convergent).  Extra targets
    carry their center's target normal.  targets_per_center = "mixed:M"
    draws each center's count log-uniformly from 1..M (a mix of centers
    on both sides of the conventional path's break-even)."""
    g, mu, tree = torus(nu, nv, seed_offset=seed_offset, n_max=n_max)
    rng = np.random.default_rng(BASE_SEED + 5 + seed_offset)
    n = g.n_ctr
    if isinstance(targets_per_center, str) and targets_per_center.startswith("mixed:"):
        top = int(targets_per_center.split(":")[1])
        counts = np.clip(np.round(np.exp(rng.uniform(0.0, np.log(top), n))), 1, top).astype(np.int64)
    else:
        counts = np.full(n, int(targets_per_center), np.int64)
    extra = counts - 1
    if extra.sum() > 0:
        c = np.repeat(np.arange(n, dtype=np.int32), extra)
        rho = np.linalg.norm(g.tgt_xyz - g.ctr_xyz, axis=0)        # one target per center, in order
        v = rng.standard_normal((len(c), 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        r = rho[c] * rng.uniform(0.0, 1.0, len(c)) ** (1.0 / 3.0)
        t = g.ctr_xyz[:, c].T + r[:, None] * v
        g.tgt_xyz = np.ascontiguousarray(np.concatenate([g.tgt_xyz, t.T], axis=1))
        g.tgt_center = np.concatenate([g.tgt_center, c])
        g.tgt_normal = np.ascontiguousarray(np.concatenate([g.tgt_normal, g.tgt_normal[:, c]], axis=1))
    g.meta.update(name=f"torus-{nu}x{nv}-tpc{targets_per_center}", targets_per_center=targets_per_center)
    return g, mu, tree


def torus_points(nu=256, nv=96):
    """The torus recipe's raw list-building inputs: sources (N, 3), QBX centers
    (M, 3) and their radii (M,), before the octree orders them."""
    V, F = mesh.torus(nu, nv, 1.0, 0.35)
    F = mesh.orient_outward(V, F, _torus_core)
    xyz, w, nrm, h = _surface_nodes(V, F)
    one = np.ones(len(xyz))
    C, Rr, T, Tn, node = mesh.centers_and_targets(xyz, nrm, h, [one, -one])
    return xyz, C, Rr


def urchin_radius(k, dirs):
    """The urchin gamma_k of Sec. 5.1: r_k = 0.2 + (Re Y_k^{floor(k/2)} - m_k)
    / (M_k - m_k) at unit directions dirs (N, 3), with M_k, m_k the extrema
    of Re Y_k^{floor(k/2)} over the sphere (taken on a 1201 x 2400 grid in
    (theta, phi) and the given directions).  P_k^m is taken without the
    Condon-Shortley phase; the spherical-harmonic normalisation cancels."""
    m = k // 2
    th, ph = np.meshgrid(np.linspace(0.0, np.pi, 1201), np.linspace(0.0, 2 * np.pi, 2400, endpoint=False))
    grid = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=-1).reshape(-1, 3)
    yg = dens.real_sph_harm(k, m, grid)
    y = dens.real_sph_harm(k, m, dirs)
    hi, lo = max(yg.max(), y.max()), min(yg.min(), y.min())
    return 0.2 + (y - lo) / (hi - lo)


def urchin_points(k=8, subdiv=5):
    """Raw list-building inputs on the urchin gamma_k as flat triangles: an
    icosphere subdivided subdiv times, each vertex moved radially to r_k;
    6 nodes per triangle, two QBX centers per node (one each side)."""
    V, F = mesh.icosphere(subdiv)
    dirs = V / np.linalg.norm(V, axis=1, keepdims=True)
    V = dirs * urchin_radius(k, dirs)[:, None]
    F = mesh.orient_outward(V, F, lambda c: np.zeros_like(c))
    xyz, w, nrm, h = _surface_nodes(V, F)
    one = np.ones(len(xyz))
    C, Rr, T, Tn, node = mesh.centers_and_targets(xyz, nrm, h, [one, -one])
    return xyz, C, Rr


def torus_helmholtz(nu=444, nv=166, k=10.0, seed_offset=0, n_max=64):
    """Helmholtz SLP workload on the refined torus with octree lists."""
    rng = np.random.default_rng(BASE_SEED + 2 + seed_offset)
    V, F = mesh.torus(nu, nv, 1.0, 0.35)
    F = mesh.orient_outward(V, F, _torus_core)
    xyz, w, nrm, h = _surface_nodes(V, F)
    one = np.ones(len(xyz))
    g, tree = _geometry_octree(xyz, w, nrm, h, [one, -one], n_max=n_max)
    g.meta.update(name=f"torus-{nu}x{nv}", kernel="helmholtz", p=12, k=k)
    return g, dens.plane_wave_density(g.src_xyz.T, k, rng), tree


def _torus_core(c, R=1.0):
    """Nearest point of the torus core circle (radius R in the xy-plane)."""
    rho = np.linalg.norm(c[:, :2], axis=1, keepdims=True)
    core = np.zeros_like(c)
    core[:, :2] = R * c[:, :2] / np.maximum(rho, 1e-300)
    return core


def ellipsoid(freq, axes, list_len_range=(50, 800), rng=None, seed_offset=0):
    """One ellipsoid of the batched workload: geodesic sphere of frequency freq
    (20 freq^2 triangles, 120 freq^2 sources) scaled by axes, one center per
    node (alternating sides).  Each center is its own group and lists one
    window of consecutive sources in Morton order (spatially local) around its
    node, of log-uniform length in list_len_range."""
    rng = rng if rng is not None else np.random.default_rng(BASE_SEED + 3 + seed_offset)
    V, F = mesh.geodesic_sphere(freq)
    V = V * np.asarray(axes)[None, :]
    F = mesh.orient_outward(V, F, lambda c: np.zeros_like(c))
    xyz, w, nrm, h = _surface_nodes(V, F)
    n = len(xyz)
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    C, Rr, T, Tn, node = mesh.centers_and_targets(xyz, nrm, h, [sign])
    lo, hi = np.log(list_len_range[0]), np.log(list_len_range[1])
    counts = np.minimum(np.exp(rng.uniform(lo, hi, len(C))).astype(np.int64), n)
    rb = np.clip(node - counts // 2, 0, None)
    rb = np.minimum(rb, n - counts).astype(np.int32)
    re = (rb + counts).astype(np.int32)
    m = len(C)
    g = Geometry(np.ascontiguousarray(xyz.T), w, np.ascontiguousarray(nrm.T),
                 np.ascontiguousarray(C.T), Rr, np.ascontiguousarray(T.T),
                 np.arange(m, dtype=np.int32), np.ascontiguousarray(Tn.T),
                 np.arange(m, dtype=np.int32), np.arange(m + 1, dtype=np.int64), rb, re)
    g.meta.update(name=f"ellipsoid-f{freq}", kernel="laplace")
    return g, dens.sphere_density(xyz, rng)


def ellipsoid_batch(n_surfaces=64, min_src=1000, max_src=200000, seed_offset=0):
    """The batched workload: n_surfaces seeded ellipsoids with log-uniform sizes
    (120 f^2 sources for frequency f) and p uniform in {5, 7, 9}."""
    rng = np.random.default_rng(BASE_SEED + 3 + seed_offset)
    out = []
    for _ in range(n_surfaces):
        axes = rng.uniform(0.5, 2.0, 3)
        target = np.exp(rng.uniform(np.log(min_src), np.log(max_src)))
        freq = int(max(3, min(40, round(np.sqrt(target / 120.0)))))
        p = int(rng.choice([5, 7, 9]))
        g, mu = ellipsoid(freq, axes, rng=rng)
        g.meta["p"] = p
        out.append((g, mu))
    return out


def serving_geometries(n=16, min_src=5000, max_src=300000, seed_offset=0):
    """The resident geometries of the serving workload: n surfaces with
    log-uniform source counts in [min_src, max_src], cycling through spheres
    and ellipsoids (one center per node, per-center Morton-window lists) and
    tori (two centers per node, octree lists)."""
    rng = np.random.default_rng(BASE_SEED + 4 + seed_offset)
    out = []
    for i in range(n):
        target = float(np.exp(rng.uniform(np.log(min_src), np.log(max_src))))
        kind = i % 3
        if kind == 2:                                  # torus: 12 nu nv sources, nv ~ 3 nu / 8
            nu = int(max(16, round(np.sqrt(target / 12.0 * 8.0 / 3.0))))
            nv = int(max(6, round(3 * nu / 8)))
            g, _, _ = torus(nu, nv, seed_offset=100 + i)
        else:
            freq = int(max(3, round(np.sqrt(target / 120.0))))
            axes = np.ones(3) if kind == 0 else rng.uniform(0.5, 2.0, 3)
            g, _ = ellipsoid(freq, axes, rng=rng)
        g.meta["serving_index"] = i
        out.append(g)
    return out
