"""Flat-triangle surfaces, interior quadrature nodes, QBX centers and targets.

Stand-ins for the paper's curvilinear test geometries (Sec. 5: urchins, the
torus grid, the plane): the meshes here are flat triangles with six interior
nodes each, centers placed along the node normals at distance h/2
(h = sqrt(triangle area)), ball radius h/2, and one target per center at half
the radius from it, on the segment towards the surface (cf. Fig. 1, where QBX
targets on the surface are served by centers placed off it).
"""
import numpy as np

# Six-point, degree-4 symmetric rule on a triangle (Dunavant 1985 / Strang-Fix):
# two barycentric orbits (a, a, 1-2a) and (b, b, 1-2b).  Weights are fractions
# of the triangle area; the workloads use equal weights area/6 per node.
RULE6_A = 0.445948490915965
RULE6_B = 0.091576213509771
RULE6_WA = 0.223381589678011
RULE6_WB = 0.109951743655322


def rule6_barycentric():
    """(6, 3) barycentric coordinates and (6,) exact weights (summing to 1)."""
    a, b = RULE6_A, RULE6_B
    bary = np.array([[a, a, 1 - 2 * a], [a, 1 - 2 * a, a], [1 - 2 * a, a, a],
                     [b, b, 1 - 2 * b], [b, 1 - 2 * b, b], [1 - 2 * b, b, b]])
    w = np.array([RULE6_WA] * 3 + [RULE6_WB] * 3)
    return bary, w


# ------------------------------------------------------------------ surfaces

def icosahedron():
    t = (1.0 + 5 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def geodesic_sphere(freq):
    """Unit sphere: every icosahedron face split into freq^2 flat triangles,
    vertices projected to the sphere (20 freq^2 triangles)."""
    V, F = icosahedron()
    verts = {}
    out_v, out_f = [], []

    def vid(p):
        key = tuple(np.round(p, 12))
        if key not in verts:
            verts[key] = len(out_v)
            out_v.append(p)
        return verts[key]

    for a, b, c in F:
        A, B, C = V[a], V[b], V[c]
        grid = {}
        for i in range(freq + 1):
            for j in range(freq + 1 - i):
                p = A + (B - A) * (i / freq) + (C - A) * (j / freq)
                grid[i, j] = vid(p / np.linalg.norm(p))
        for i in range(freq):
            for j in range(freq - i):
                out_f.append([grid[i, j], grid[i + 1, j], grid[i, j + 1]])
                if i + j + 1 < freq:
                    out_f.append([grid[i + 1, j], grid[i + 1, j + 1], grid[i, j + 1]])
    return np.array(out_v), np.array(out_f, dtype=np.int64)


def icosphere(subdiv):
    """Unit sphere from the icosahedron by `subdiv` rounds of 1-to-4 splitting."""
    V, F = icosahedron()
    V = list(V)
    for _ in range(subdiv):
        mid = {}

        def m(i, j):
            key = (min(i, j), max(i, j))
            if key not in mid:
                p = V[i] + V[j]
                V.append(p / np.linalg.norm(p))
                mid[key] = len(V) - 1
            return mid[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        F = np.array(nf, dtype=np.int64)
    return np.array(V), F


def torus(nu, nv, R=1.0, r=0.35):
    """Torus (R + r cos v) (cos u, sin u) + r sin v e_z on an nu x nv quad grid,
    each quad split into two triangles (2 nu nv triangles)."""
    u = 2 * np.pi * np.arange(nu) / nu
    v = 2 * np.pi * np.arange(nv) / nv
    U, Vv = np.meshgrid(u, v, indexing="ij")
    X = np.stack([(R + r * np.cos(Vv)) * np.cos(U), (R + r * np.cos(Vv)) * np.sin(U),
                  r * np.sin(Vv)], axis=-1).reshape(-1, 3)
    idx = np.arange(nu * nv).reshape(nu, nv)
    i0, j0 = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a = idx[i0, j0]
    b = idx[(i0 + 1) % nu, j0]
    c = idx[(i0 + 1) % nu, (j0 + 1) % nv]
    d = idx[i0, (j0 + 1) % nv]
    F = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3),
                        np.stack([a, c, d], -1).reshape(-1, 3)])
    return X, F


def orient_outward(V, F, inside_point_fn):
    """Flip faces so that the face normal points away from inside_point_fn(centroid)."""
    P = V[F]
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    cen = P.mean(axis=1)
    flip = np.einsum("ij,ij->i", n, cen - inside_point_fn(cen)) < 0
    F = F.copy()
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


# ------------------------------------------------------------- discretisation

def nodes_on_triangles(V, F):
    """Six interior nodes per flat triangle.  Returns xyz (n,3), equal weights
    area/6 (n,), unit face normals (n,3), h = sqrt(area) per node (n,), and the
    exact rule weights (n,) for reference."""
    bary, wexact = rule6_barycentric()
    P = V[F]                                       # (nf, 3, 3)
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nrm = cr / (2 * area[:, None])
    xyz = np.einsum("qk,fkd->fqd", bary, P).reshape(-1, 3)
    w = np.repeat(area / 6.0, 6)
    wex = (area[:, None] * wexact[None, :]).reshape(-1)
    normals = np.repeat(nrm, 6, axis=0)
    h = np.repeat(np.sqrt(area), 6)
    return xyz, w, normals, h, wex


def morton_order(xyz, bits=20):
    """Permutation sorting points along a Morton (Z-order) curve."""
    lo = xyz.min(axis=0)
    span = max(float((xyz.max(axis=0) - lo).max()), 1e-300)
    q = np.clip(((xyz - lo) / span * (2 ** bits - 1)).astype(np.uint64), 0, 2 ** bits - 1)
    code = np.zeros(len(xyz), dtype=np.uint64)
    for bit in range(bits):
        for d in range(3):
            code |= ((q[:, d] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(3 * bit + d)
    return np.argsort(code, kind="stable")


def centers_and_targets(xyz, normals, h, signs):
    """One center per (node, sign) at node + sign h/2 n, radius h/2, and one
    target at half the radius from the center towards the node.  `signs` is a
    list of per-node sign arrays; centers are emitted sign-block by sign-block."""
    C, Rr, T, Tn, node = [], [], [], [], []
    for s in signs:
        s = np.asarray(s, dtype=np.float64)[:, None]
        c = xyz + s * (h[:, None] / 2) * normals
        r = h / 2
        t = c - s * (r[:, None] / 2) * normals
        C.append(c)
        Rr.append(r)
        T.append(t)
        Tn.append(normals)
        node.append(np.arange(len(xyz)))
    return (np.concatenate(C), np.concatenate(Rr), np.concatenate(T), np.concatenate(Tn),
            np.concatenate(node))
