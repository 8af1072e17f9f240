"""Seeded generators for hex spectral-element meshes, query points and fields.

Layouts produced here are the ones the C-ABI consumes:
  coords  float64 [3][E][n^3]   node (i,j,k) of element e at i + n*(j + n*k)
  sub     int32   [E]           subdomain (session) id of each element
  dist    float64 [E][n^3]      nodal distance-to-boundary field D^k (closed form)
  pts     float64 [3][P]        query points
  qsess   int32   [P]           session tag of each query (-1 = search all)
  fields  float64 [F][E][n^3]   nodal values of the fields to interpolate

Node placement uses numpy's own Legendre-root routine for the reference grid,
independent of the GLL code in the oracle and in the CUDA library; a mesh is
fully defined by its node coordinates, so a last-bit difference in where the
generator put a node does not matter to either side.

Workloads (mesh sizes, perturbations, query mixes) follow the five configurations
the library is measured on: a 4x4x4 deformed cube (N=7), a box + annular cylinder
overlap pair, a 32^3 deformed cube with 1e7 uniform + 1e5 near-face points, a
batch of 64 deformed boxes of mixed E and N, and a served three-subdomain overlap
(box + two rotated annular cylinders).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "Mesh", "Queries", "reference_grid", "box_mesh", "annulus_mesh", "concat_meshes",
    "box_distance", "annulus_distance", "uniform_points", "near_face_points",
    "boundary_face_nodes", "field_u", "sine_product_field", "random_poly_field",
    "cube4_small", "box_annulus", "deformed_cube", "instance_batch", "box_two_annuli", "poisson_requests",
    "tiny_overlap", "spiral_element", "reference_poly_field", "rigid_motion",
    "quad_mesh", "ring_mesh", "rect_distance", "uniform_points_2d", "edge_points_2d", "field_u_2d",
    "reference_poly_field_2d", "tiny_overlap_2d", "walsh_2d",
]


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclass
class Mesh:
    coords: np.ndarray                    # [3][E][n^3] float64
    N: int
    sub: np.ndarray                       # [E] int32
    dist: Optional[np.ndarray] = None     # [E][n^3] float64 or None
    name: str = ""

    @property
    def E(self) -> int:
        return int(self.coords.shape[1])

    @property
    def n(self) -> int:
        return self.N + 1


@dataclass
class Queries:
    pts: np.ndarray                       # [3][P] float64
    qsess: Optional[np.ndarray] = None    # [P] int32 or None
    fields: Optional[np.ndarray] = None   # [F][E][n^3] float64
    info: dict = field(default_factory=dict)

    @property
    def P(self) -> int:
        return int(self.pts.shape[1])


# ----------------------------------------------------------------------------
# reference grid and meshes
# ----------------------------------------------------------------------------
def reference_grid(N: int) -> np.ndarray:
    """Gauss-Lobatto-Legendre abscissae on [-1,1] for node placement, via
    numpy's Legendre root finder (endpoints plus roots of P_N')."""
    if N < 1:
        raise ValueError("N >= 1")
    if N == 1:
        return np.array([-1.0, 1.0])
    inner = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real)
    x = np.concatenate([[-1.0], inner, [1.0]])
    x = 0.5 * (x - x[::-1])            # exact antisymmetry
    if N % 2 == 0:
        x[N // 2] = 0.0
    return x


def _axis_nodes(m: int, a: float, b: float, xi: np.ndarray) -> np.ndarray:
    """[m][n] node coordinates along one axis for m equal elements on [a,b].
    The end nodes of neighbouring elements come from the same expression, so
    shared nodes are bit-identical."""
    t = (np.arange(m)[:, None] + 0.5 * (xi[None, :] + 1.0)) / m
    g = a + (b - a) * t
    g[:, 0] = a + (b - a) * (np.arange(m) / m)
    g[:, -1] = a + (b - a) * (np.arange(1, m + 1) / m)
    return g


def box_mesh(shape, N: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
             amp_frac: float = 0.0) -> np.ndarray:
    """Hex mesh of the box [lo,hi] with shape=(ex,ey,ez) elements of order N,
    element e = ei + ex*(ej + ey*ek).  With amp_frac > 0 every node not on the
    box boundary is moved by the same scalar d = amp_frac*h*sin(2 pi x')
    sin(2 pi y') sin(2 pi z') added to each of its three coordinates, where
    x' = (x-lo)/(hi-lo) is the undeformed position scaled to the unit cube and
    h the smallest element width.  Returns coords [3][E][n^3]."""
    ex, ey, ez = (int(v) for v in shape)
    xi = reference_grid(N)
    n = N + 1
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    gx = _axis_nodes(ex, lo[0], hi[0], xi)
    gy = _axis_nodes(ey, lo[1], hi[1], xi)
    gz = _axis_nodes(ez, lo[2], hi[2], xi)
    shp = (ez, ey, ex, n, n, n)
    X = np.broadcast_to(gx[None, None, :, None, None, :], shp)
    Y = np.broadcast_to(gy[None, :, None, None, :, None], shp)
    Z = np.broadcast_to(gz[:, None, None, :, None, None], shp)
    E = ex * ey * ez
    coords = np.empty((3, E, n ** 3), dtype=np.float64)
    coords[0] = X.reshape(E, n ** 3)
    coords[1] = Y.reshape(E, n ** 3)
    coords[2] = Z.reshape(E, n ** 3)
    if amp_frac:
        h = float(np.min((hi - lo) / np.array([ex, ey, ez])))
        A = amp_frac * h
        u = (coords[0] - lo[0]) / (hi[0] - lo[0])
        v = (coords[1] - lo[1]) / (hi[1] - lo[1])
        w = (coords[2] - lo[2]) / (hi[2] - lo[2])
        d = A * np.sin(2 * np.pi * u) * np.sin(2 * np.pi * v) * np.sin(2 * np.pi * w)
        on_bnd = ((coords[0] == lo[0]) | (coords[0] == hi[0]) |
                  (coords[1] == lo[1]) | (coords[1] == hi[1]) |
                  (coords[2] == lo[2]) | (coords[2] == hi[2]))
        d[on_bnd] = 0.0
        coords += d[None]
    return coords


def _rotation(rx_deg: float = 0.0, ry_deg: float = 0.0) -> np.ndarray:
    """R = Ry(ry) @ Rx(rx)."""
    a, b = math.radians(rx_deg), math.radians(ry_deg)
    Rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    return Ry @ Rx


def annulus_mesh(n_az: int, n_rad: int, n_ax: int, N: int, r_in: float, r_out: float,
                 z0: float, z1: float, center=(0.0, 0.0, 0.0), rot=(0.0, 0.0)):
    """Annular cylinder r_in <= rho <= r_out, z0 <= z <= z1 (local frame) meshed
    n_az x n_rad x n_ax, nodes placed by the exact polar map with GLL-spaced
    (rho, theta, z) inside uniform element intervals, theta_0 = 0.  Reference
    directions: r -> radial, s -> azimuthal, t -> axial (positive Jacobian);
    element e = er + n_rad*(ea + n_az*ez).  The local frame is rotated by
    R = Ry(rot[1]) Rx(rot[0]) and translated to `center`.
    Returns (coords [3][E][n^3], local (rho, zloc) arrays [E][n^3])."""
    xi = reference_grid(N)
    n = N + 1
    grho = _axis_nodes(n_rad, r_in, r_out, xi)
    gth = _axis_nodes(n_az, 0.0, 2.0 * np.pi, xi)
    gth[-1, -1] = 0.0                       # wrap: last node is the first
    gz = _axis_nodes(n_ax, z0, z1, xi)
    shp = (n_ax, n_az, n_rad, n, n, n)
    RHO = np.broadcast_to(grho[None, None, :, None, None, :], shp)
    TH = np.broadcast_to(gth[None, :, None, None, :, None], shp)
    ZZ = np.broadcast_to(gz[:, None, None, :, None, None], shp)
    E = n_az * n_rad * n_ax
    rho = np.ascontiguousarray(RHO.reshape(E, n ** 3))
    th = TH.reshape(E, n ** 3)
    zl = np.ascontiguousarray(ZZ.reshape(E, n ** 3))
    xl = rho * np.cos(th)
    yl = rho * np.sin(th)
    R = _rotation(*rot)
    c = np.asarray(center, dtype=np.float64)
    coords = np.empty((3, E, n ** 3), dtype=np.float64)
    for a in range(3):
        coords[a] = c[a] + R[a, 0] * xl + R[a, 1] * yl + R[a, 2] * zl
    return coords, rho, zl


def concat_meshes(parts: List[np.ndarray], N: int, subs: List[int],
                  dists: Optional[List[np.ndarray]] = None, name: str = "") -> Mesh:
    coords = np.concatenate(parts, axis=1)
    sub = np.concatenate([np.full(p.shape[1], s, dtype=np.int32) for p, s in zip(parts, subs)])
    dist = None if dists is None else np.concatenate(dists, axis=0)
    return Mesh(coords=np.ascontiguousarray(coords), N=N, sub=sub, dist=dist, name=name)


def box_distance(coords: np.ndarray, lo, hi) -> np.ndarray:
    """Closed-form distance of each node of an undeformed box mesh to the box
    boundary: min over the six faces.  [E][n^3]."""
    d = None
    for a in range(3):
        for v in (coords[a] - lo[a], hi[a] - coords[a]):
            d = v.copy() if d is None else np.minimum(d, v)
    return np.maximum(d, 0.0)


def annulus_distance(rho: np.ndarray, zl: np.ndarray, r_in, r_out, z0, z1) -> np.ndarray:
    """Closed-form distance of an annular-cylinder node to the cylinder's
    boundary: min(rho-r_in, r_out-rho, z-z0, z1-z) in the local frame."""
    d = np.minimum(np.minimum(rho - r_in, r_out - rho), np.minimum(zl - z0, z1 - zl))
    return np.maximum(d, 0.0)


# ----------------------------------------------------------------------------
# queries and fields
# ----------------------------------------------------------------------------
def uniform_points(P: int, seed: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> np.ndarray:
    """P points uniform in [lo,hi), drawn as rng.random((P,3)); returns [3][P]."""
    rng = np.random.default_rng(seed)
    u = rng.random((P, 3))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return np.ascontiguousarray((lo + (hi - lo) * u).T)


def near_face_points(coords: np.ndarray, N: int, M: int, seed: int,
                     lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> np.ndarray:
    """M points within 1e-9 of element faces of a (deformed) box mesh.

    Each point starts at a face-interior GLL node of a random element and face
    (node indices 1..N-1 on the face, so the start lies on exactly one face and
    away from edges) and is moved along the face's nominal axis by
    side*10^U(-11,-9) for 90% of the points and by exactly 0 for the other 10%.
    A point pushed outside the box is mirrored back inside.  Returns [3][M]."""
    if N < 2:
        raise ValueError("near-face points need N >= 2")
    rng = np.random.default_rng(seed)
    E = coords.shape[1]
    n = N + 1
    e = rng.integers(0, E, size=M)
    f = rng.integers(0, 6, size=M)
    a = rng.integers(1, N, size=M)
    b = rng.integers(1, N, size=M)
    mag = np.where(rng.random(M) < 0.9, 10.0 ** rng.uniform(-11.0, -9.0, size=M), 0.0)
    side = np.where(rng.random(M) < 0.5, -1.0, 1.0)
    end = np.where(f % 2 == 0, 0, N)
    ax = f // 2
    i = np.where(ax == 0, end, a)
    j = np.where(ax == 0, a, np.where(ax == 1, end, b))
    k = np.where(ax == 2, end, b)
    idx = i + n * (j + n * k)
    p = coords[:, e, idx].copy()
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    for c in range(3):
        sel = ax == c
        q = p[c, sel] + side[sel] * mag[sel]
        out = (q < lo[c]) | (q > hi[c])
        q[out] = p[c, sel][out] - side[sel][out] * mag[sel][out]
        p[c, sel] = q
    return np.ascontiguousarray(p)


def boundary_face_nodes(coords: np.ndarray, N: int, shape, faces="all") -> np.ndarray:
    """Deduplicated GLL nodes on the outer faces of a structured block mesh with
    element grid shape=(m0,m1,m2) in reference directions (r,s,t).  `faces` is
    'all' or a list of (axis, end) pairs, end 0 = low, 1 = high.  Returns [3][Q]."""
    n = N + 1
    m = [int(v) for v in shape]
    E = m[0] * m[1] * m[2]
    C = coords.reshape(3, m[2], m[1], m[0], n, n, n)    # [3][e2][e1][e0][k][j][i]
    if faces == "all":
        faces = [(a, s) for a in range(3) for s in (0, 1)]
    chunks = []
    for ax, s in faces:
        sl = [slice(None)] * 7
        sl[0] = slice(None)
        eidx = 0 if s == 0 else m[ax] - 1
        nidx = 0 if s == 0 else N
        sl[3 - ax] = eidx              # element axis: e0 at 3, e1 at 2, e2 at 1
        sl[6 - ax] = nidx              # node axis: i at 6, j at 5, k at 4
        chunks.append(C[tuple(sl)].reshape(3, -1))
    allp = np.concatenate(chunks, axis=1).T
    uniq = np.unique(allp, axis=0)
    assert E == coords.shape[1]
    return np.ascontiguousarray(uniq.T)


def field_u(coords: np.ndarray) -> np.ndarray:
    """u = sin(pi x) cos(pi y) exp(z) at the nodes.  [E][n^3]."""
    return np.sin(np.pi * coords[0]) * np.cos(np.pi * coords[1]) * np.exp(coords[2])


def sine_product_field(coords: np.ndarray, seed: int) -> np.ndarray:
    """sin(a0 x + b0) sin(a1 y + b1) sin(a2 z + b2), a ~ U[1,3]*pi, b ~ U[0,2pi)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(1.0, 3.0, size=3) * np.pi
    b = rng.uniform(0.0, 2 * np.pi, size=3)
    return (np.sin(a[0] * coords[0] + b[0]) * np.sin(a[1] * coords[1] + b[1]) *
            np.sin(a[2] * coords[2] + b[2]))


def _monomials(deg: int):
    return [(i, j, k) for i in range(deg + 1) for j in range(deg + 1 - i)
            for k in range(deg + 1 - i - j)]


def random_poly_field(coords: np.ndarray, deg: int, rng: np.random.Generator):
    """Random polynomial of total degree <= deg in (x,y,z), coefficients
    U[-1,1]; returns (nodal values [E][n^3], list of (coef, (i,j,k)))."""
    terms = [(rng.uniform(-1.0, 1.0), m) for m in _monomials(deg)]
    v = np.zeros(coords.shape[1:], dtype=np.float64)
    for c, (i, j, k) in terms:
        v += c * coords[0] ** i * coords[1] ** j * coords[2] ** k
    return v, terms


def reference_poly_field(N: int, E: int, seed: int):
    """Nodal values u_ijk = p(xi_i, xi_j, xi_k) of a random polynomial p in
    Q_N (degree <= N in each reference variable), the same p on every element.
    Returns (values [E][n^3], coefficient tensor c[a,b,c] for r^a s^b t^c)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1.0, 1.0, size=(N + 1, N + 1, N + 1))
    xi = reference_grid(N)
    n = N + 1
    V = np.vander(xi, N + 1, increasing=True)         # V[i,a] = xi_i^a
    vals = np.einsum("ia,jb,kc,abc->kji", V, V, V, c).reshape(n ** 3)
    return np.ascontiguousarray(np.broadcast_to(vals, (E, n ** 3))), c


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------
def cube4_small():
    """Unit cube 4x4x4 hex, N=7, interior nodes displaced by 0.05 h sin sin sin,
    1e4 uniform points (seed 0), field u = sin(pi x)cos(pi y)exp(z)."""
    N = 7
    coords = box_mesh((4, 4, 4), N, amp_frac=0.05)
    mesh = Mesh(coords=coords, N=N, sub=np.zeros(coords.shape[1], np.int32), name="cube4-N7")
    pts = uniform_points(10 ** 4, seed=0)
    fields = field_u(coords)[None]
    return mesh, Queries(pts=pts, fields=np.ascontiguousarray(fields), info={"P": pts.shape[1]})


# the azimuthal direction of an annulus is periodic: only radial and axial faces bound it
ANNULUS_FACES = [(0, 0), (0, 1), (2, 0), (2, 1)]

BOX_ANNULUS_BOX = dict(lo=(0.0, 0.0, 0.0), hi=(2.0, 1.0, 1.0))
BOX_ANNULUS_CYL = dict(r_in=0.15, r_out=0.35, z0=0.0, z1=1.0, center=(1.0, 0.5, 0.0))


def box_annulus(n_az=32, n_rad=4, n_ax=8, box_shape=(16, 8, 8), N=7, margin=0.0):
    """Box [0,2]x[0,1]^2 (16x8x8, session 0) overlapped by the annular cylinder
    rho in [0.15,0.35] around (1,0.5), z in [0,1] (32 az x 4 rad x 8 ax,
    session 1), N=7.  Queries: the deduplicated boundary GLL nodes of each
    subdomain lying in the other subdomain's exact geometry, tagged with their
    own session (every cylinder boundary node; box z-face nodes with
    r_in - margin <= rho <= r_out + margin).  Four fields u,v,w,p: random
    total-degree <= 5 polynomials (seed 1).  D^k in closed form."""
    cb = box_mesh(box_shape, N, **BOX_ANNULUS_BOX)
    cc, rho, zl = annulus_mesh(n_az, n_rad, n_ax, N, BOX_ANNULUS_CYL["r_in"], BOX_ANNULUS_CYL["r_out"],
                               BOX_ANNULUS_CYL["z0"], BOX_ANNULUS_CYL["z1"], center=BOX_ANNULUS_CYL["center"])
    db = box_distance(cb, BOX_ANNULUS_BOX["lo"], BOX_ANNULUS_BOX["hi"])
    dc = annulus_distance(rho, zl, BOX_ANNULUS_CYL["r_in"], BOX_ANNULUS_CYL["r_out"], BOX_ANNULUS_CYL["z0"], BOX_ANNULUS_CYL["z1"])
    mesh = concat_meshes([cb, cc], N, [0, 1], [db, dc], name="box+annulus-N7")
    qc = boundary_face_nodes(cc, N, (n_rad, n_az, n_ax), faces=ANNULUS_FACES)
    qb = boundary_face_nodes(cb, N, box_shape, faces=[(2, 0), (2, 1)])
    rb = np.hypot(qb[0] - 1.0, qb[1] - 0.5)
    keep = (rb >= BOX_ANNULUS_CYL["r_in"] - margin) & (rb <= BOX_ANNULUS_CYL["r_out"] + margin)
    qb = qb[:, keep]
    pts = np.ascontiguousarray(np.concatenate([qb, qc], axis=1))
    qsess = np.concatenate([np.zeros(qb.shape[1], np.int32), np.ones(qc.shape[1], np.int32)])
    rng = np.random.default_rng(1)
    fields = np.stack([random_poly_field(mesh.coords, 5, rng)[0] for _ in range(4)])
    return mesh, Queries(pts=pts, qsess=qsess, fields=fields,
                         info={"P_box": int(qb.shape[1]), "P_cyl": int(qc.shape[1])})


def deformed_cube(ne=32, P_uniform=10 ** 7, P_face=10 ** 5, N=7, with_fields=True):
    """ne^3 deformed hex (amplitude 0.1 h), N=7; P_uniform uniform points
    (seed 0) followed by P_face near-face points (seed 1); five fields
    u (as in cube4_small) and sine products with seeds 2-5."""
    coords = box_mesh((ne, ne, ne), N, amp_frac=0.1)
    mesh = Mesh(coords=coords, N=N, sub=np.zeros(coords.shape[1], np.int32),
                name=f"cube{ne}-N{N}")
    pu = uniform_points(P_uniform, seed=0)
    pf = near_face_points(coords, N, P_face, seed=1) if P_face else np.zeros((3, 0))
    pts = np.ascontiguousarray(np.concatenate([pu, pf], axis=1))
    fields = None
    if with_fields:
        fields = np.empty((5,) + coords.shape[1:], dtype=np.float64)
        fields[0] = field_u(coords)
        for s in range(4):
            fields[1 + s] = sine_product_field(coords, seed=2 + s)
    return mesh, Queries(pts=pts, fields=fields, info={"P_uniform": P_uniform, "P_face": P_face})


def instance_batch(n_inst=64, seed=3, E_range=(64, 8192), P_range=(10 ** 3, 10 ** 6),
            Ns=(5, 7, 9), scale=1.0):
    """n_inst independent deformed unit-cube instances (amplitude 0.05 h):
    E ~ logU(E_range) rounded to near-cubic ex*ey*ez, N uniform in Ns,
    P ~ logU(P_range) uniform points, one field u.  `scale` multiplies the
    point counts (for reduced-size tests).  Returns a list of (Mesh, Queries)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        Et = math.exp(rng.uniform(math.log(E_range[0]), math.log(E_range[1])))
        N = int(rng.choice(Ns))
        P = int(round(math.exp(rng.uniform(math.log(P_range[0]), math.log(P_range[1])))))
        ex = max(1, int(round(Et ** (1.0 / 3.0))))
        ey = max(1, int(round(math.sqrt(Et / ex))))
        ez = max(1, int(round(Et / (ex * ey))))
        coords = box_mesh((ex, ey, ez), N, amp_frac=0.05)
        mesh = Mesh(coords=coords, N=N, sub=np.zeros(coords.shape[1], np.int32),
                    name=f"inst{i}-{ex}x{ey}x{ez}-N{N}")
        Pi = max(1, int(round(P * scale)))
        pts = uniform_points(Pi, seed=1000 + i)
        out.append((mesh, Queries(pts=pts, fields=field_u(coords)[None].copy(),
                                  info={"shape": (ex, ey, ez)})))
    return out


SERVED_BOX = dict(lo=(0.0, 0.0, 0.0), hi=(2.0, 1.0, 1.0))
SERVED_CYLS = [dict(center=(0.85, 0.5, 0.5), rot=(15.0, 0.0)),
        dict(center=(1.15, 0.5, 0.5), rot=(0.0, -15.0))]


def box_two_annuli(box_shape=(80, 40, 40), cyl_shape=(64, 8, 64), N=7):
    """Background box [0,2]x[0,1]^2 (session 0) + two annular cylinders
    rho in [0.15,0.35], length 0.6, (az,rad,ax) = cyl_shape, centred at
    (0.85,0.5,0.5) with axis rotated +15 deg about x (session 1) and at
    (1.15,0.5,0.5) rotated -15 deg about y (session 2).  D^k in closed form.
    Returns (Mesh, [interface node arrays [3][Q] per cylinder])."""
    parts, dists, iface = [], [], []
    cb = box_mesh(box_shape, N, **SERVED_BOX)
    parts.append(cb)
    dists.append(box_distance(cb, SERVED_BOX["lo"], SERVED_BOX["hi"]))
    for c in SERVED_CYLS:
        cc, rho, zl = annulus_mesh(cyl_shape[0], cyl_shape[1], cyl_shape[2], N, 0.15, 0.35,
                                   -0.3, 0.3, center=c["center"], rot=c["rot"])
        parts.append(cc)
        dists.append(annulus_distance(rho, zl, 0.15, 0.35, -0.3, 0.3))
        iface.append(boundary_face_nodes(cc, N, (cyl_shape[1], cyl_shape[0], cyl_shape[2]),
                                         faces=ANNULUS_FACES))
    mesh = concat_meshes(parts, N, [0, 1, 2], dists, name="box+2annuli-N7")
    return mesh, iface


def poisson_requests(iface, n_req: int, seed: int = 4, size_range=(10 ** 2, 10 ** 6),
                     rate_hz: float = 100.0):
    """Poisson request stream: sizes logU(size_range); each request is 50%
    uniform points in the box (untagged, -1) and 50% cylinder interface nodes
    tagged with their cylinder's session.  Returns a list of dicts with
    't_arrive' (s), 'pts' [3][P] and 'qsess' [P]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for r in range(n_req):
        t += rng.exponential(1.0 / rate_hz)
        P = int(round(math.exp(rng.uniform(math.log(size_range[0]), math.log(size_range[1])))))
        Pu = P // 2
        Pi = P - Pu
        pu = (np.array(SERVED_BOX["lo"]) + (np.array(SERVED_BOX["hi"]) - np.array(SERVED_BOX["lo"])) *
              rng.random((Pu, 3))).T
        which = rng.integers(0, len(iface), size=Pi)
        pi = np.empty((3, Pi))
        qs = np.empty(Pi, np.int32)
        for c, nodes in enumerate(iface):
            sel = which == c
            k = rng.integers(0, nodes.shape[1], size=int(sel.sum()))
            pi[:, sel] = nodes[:, k]
            qs[sel] = c + 1
        pts = np.ascontiguousarray(np.concatenate([pu, pi], axis=1))
        qsess = np.concatenate([np.full(Pu, -1, np.int32), qs])
        reqs.append({"t_arrive": t, "pts": pts, "qsess": qsess})
    return reqs


# ----------------------------------------------------------------------------
# small hand-built cases
# ----------------------------------------------------------------------------
TINY_X = [(0.0, 1.0), (0.6, 1.6), (0.8, 2.0)]


def tiny_overlap(N=4):
    """Three overlapping boxes (sessions 0,1,2) spanning x in [0,1], [0.6,1.6],
    [0.8,2.0] and y,z in [0,1], each 2x1x1 elements split at its x-midpoint.
    D^k = min(x - a_k, b_k - x) is linear on every element, so its nodal
    interpolant is exact: delta^k(x*) is known in closed form."""
    parts, dists = [], []
    for a, b in TINY_X:
        c = box_mesh((2, 1, 1), N, lo=(a, 0.0, 0.0), hi=(b, 1.0, 1.0))
        parts.append(c)
        dists.append(np.minimum(c[0] - a, b - c[0]))
    return concat_meshes(parts, N, [0, 1, 2], dists, name="tiny-overlap")


def spiral_element(N=15):
    """One strongly curved element: an annular sector wound through 270 deg
    whose radius grows with the angle, with a sinusoidal lift in z.
    rho = 1.5 + 0.5 r + 0.3 (s+1), theta = 0.75 pi (s+1), z = t + 0.3 sin(theta).
    Returns (coords [3][1][n^3], analytic map f(r,s,t) -> x for test points)."""
    xi = reference_grid(N)
    n = N + 1
    R, S, T = np.meshgrid(xi, xi, xi, indexing="ij")       # [i][j][k]

    def amap(r, s, t):
        rho = 1.5 + 0.5 * r + 0.3 * (s + 1.0)
        th = 0.75 * np.pi * (s + 1.0)
        return np.stack([rho * np.cos(th), rho * np.sin(th), t + 0.3 * np.sin(th)])

    X = amap(R, S, T)                                       # [3][i][j][k]
    coords = np.ascontiguousarray(X.transpose(0, 3, 2, 1).reshape(3, 1, n ** 3))
    return coords, amap


def rigid_motion(coords: np.ndarray, sub: np.ndarray, moving: int, angle_deg: float = 0.0,
                 shift=(0.0, 0.0, 0.0), center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Coordinates after the elements of subdomain `moving` turn by angle_deg
    about the z axis through `center` and then shift by `shift` (a moving
    mesh); the other elements stay.  Returns a new [3][E][n^3] array."""
    out = np.array(coords, dtype=np.float64, copy=True)
    m = np.asarray(sub) == moving
    a = np.deg2rad(angle_deg)
    c, s = np.cos(a), np.sin(a)
    x = out[0, m] - center[0]
    y = out[1, m] - center[1]
    out[0, m] = center[0] + c * x - s * y + shift[0]
    out[1, m] = center[1] + s * x + c * y + shift[1]
    out[2, m] = out[2, m] + shift[2]
    return out


# ----------------------------------------------------------------------------
# 2D (quadrilateral) meshes: coords [2][E][n^2], node (i,j) at i + n*j
# ----------------------------------------------------------------------------
def quad_mesh(shape, N: int, lo=(0.0, 0.0), hi=(1.0, 1.0), amp_frac: float = 0.0) -> np.ndarray:
    """Quad mesh of the rectangle [lo,hi] with shape=(ex,ey) elements of
    order N, element e = ei + ex*ej.  With amp_frac > 0 every node not on the
    rectangle's boundary moves by d = amp_frac*h*sin(2 pi x') sin(2 pi y') in
    both coordinates (x' = (x-lo)/(hi-lo), h the smallest element width)."""
    ex, ey = (int(v) for v in shape)
    xi = reference_grid(N)
    n = N + 1
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    gx = _axis_nodes(ex, lo[0], hi[0], xi)
    gy = _axis_nodes(ey, lo[1], hi[1], xi)
    shp = (ey, ex, n, n)
    X = np.broadcast_to(gx[None, :, None, :], shp)
    Y = np.broadcast_to(gy[:, None, :, None], shp)
    E = ex * ey
    coords = np.empty((2, E, n * n), dtype=np.float64)
    coords[0] = X.reshape(E, n * n)
    coords[1] = Y.reshape(E, n * n)
    if amp_frac:
        h = float(np.min((hi - lo) / np.array([ex, ey])))
        u = (coords[0] - lo[0]) / (hi[0] - lo[0])
        v = (coords[1] - lo[1]) / (hi[1] - lo[1])
        d = amp_frac * h * np.sin(2 * np.pi * u) * np.sin(2 * np.pi * v)
        on_bnd = (coords[0] == lo[0]) | (coords[0] == hi[0]) | (coords[1] == lo[1]) | (coords[1] == hi[1])
        d[on_bnd] = 0.0
        coords += d[None]
    return coords


def ring_mesh(n_az: int, n_rad: int, N: int, r_in: float, r_out: float, center=(0.0, 0.0),
              angle0: float = 0.0):
    """Quad mesh of the annulus r_in <= rho <= r_out around `center`: n_az
    azimuthal x n_rad radial elements, element e = er + n_rad*ea, reference r
    radial, s azimuthal (counter-clockwise).  Returns (coords [2][E][n^2],
    rho [E][n^2])."""
    xi = reference_grid(N)
    n = N + 1
    rr = _axis_nodes(n_rad, r_in, r_out, xi)          # [n_rad][n]
    th = _axis_nodes(n_az, angle0, angle0 + 2 * np.pi, xi)
    th[-1, -1] = angle0                                # wrap: last node is the first
    shp = (n_az, n_rad, n, n)                          # [ea][er][j][i]
    R = np.broadcast_to(rr[None, :, None, :], shp)
    T = np.broadcast_to(th[:, None, :, None], shp)
    E = n_az * n_rad
    rho = R.reshape(E, n * n)
    t = T.reshape(E, n * n)
    coords = np.empty((2, E, n * n), dtype=np.float64)
    coords[0] = center[0] + rho * np.cos(t)
    coords[1] = center[1] + rho * np.sin(t)
    return coords, np.ascontiguousarray(rho)


def rect_distance(coords: np.ndarray, lo, hi) -> np.ndarray:
    """Closed-form distance of each node of an undeformed quad mesh to the
    rectangle's boundary.  [E][n^2]."""
    d = np.minimum(np.minimum(coords[0] - lo[0], hi[0] - coords[0]),
                   np.minimum(coords[1] - lo[1], hi[1] - coords[1]))
    return np.maximum(d, 0.0)


def uniform_points_2d(P: int, seed: int, lo=(0.0, 0.0), hi=(1.0, 1.0)) -> np.ndarray:
    """P points uniform in [lo,hi), drawn as rng.random((P,2)); returns [2][P]."""
    rng = np.random.default_rng(seed)
    u = rng.random((P, 2))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return np.ascontiguousarray((lo + (hi - lo) * u).T)


def edge_points_2d(coords: np.ndarray, N: int, M: int, seed: int) -> np.ndarray:
    """M points within 1e-9 of element edges: interior GLL nodes of random
    element edges moved along the edge's nominal normal axis by
    +-10^U(-11,-9) (90 %) or 0 (10 %).  Returns [2][M]."""
    rng = np.random.default_rng(seed)
    n = N + 1
    E = coords.shape[1]
    e = rng.integers(0, E, M)
    f = rng.integers(0, 4, M)
    a = rng.integers(1, N, M) if N > 1 else np.zeros(M, int)
    end = np.where(f % 2 == 1, N, 0)
    idx = np.where(f // 2 == 0, end + n * a, a + n * end)
    pts = np.stack([coords[0, e, idx], coords[1, e, idx]])
    off = np.where(rng.random(M) < 0.9, rng.choice([-1.0, 1.0], M) * 10.0 ** rng.uniform(-11, -9, M), 0.0)
    pts[f // 2, np.arange(M)] += off
    return np.ascontiguousarray(pts)


def field_u_2d(coords: np.ndarray) -> np.ndarray:
    """u = sin(pi x) cos(pi y) exp(x y) at the nodes of a 2D mesh."""
    return np.sin(np.pi * coords[0]) * np.cos(np.pi * coords[1]) * np.exp(coords[0] * coords[1])


def reference_poly_field_2d(N: int, E: int, seed: int):
    """Nodal values p(xi_i, xi_j) of a random p in Q_N(r, s), the same on
    every element.  Returns (values [E][n^2], coefficients c[a,b] of r^a s^b)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1.0, 1.0, size=(N + 1, N + 1))
    xi = reference_grid(N)
    V = np.vander(xi, N + 1, increasing=True)
    vals = np.einsum("ia,jb,ab->ji", V, V, c).reshape((N + 1) ** 2)
    return np.ascontiguousarray(np.broadcast_to(vals, (E, (N + 1) ** 2))), c


def tiny_overlap_2d(N=4):
    """Three overlapping rectangles (sessions 0,1,2) spanning x in TINY_X and
    y in [0,1], each 2x1 elements split at its x-midpoint; D^k = min(x - a_k,
    b_k - x) is linear on every element (closed-form delta^k)."""
    parts, dists = [], []
    for a, b in TINY_X:
        c = quad_mesh((2, 1), N, lo=(a, 0.0), hi=(b, 1.0))
        parts.append(c)
        dists.append(np.minimum(c[0] - a, b - c[0]))
    return concat_meshes(parts, N, [0, 1, 2], dists, name="tiny-overlap-2d")


def walsh_2d(N=7, n_box=16, ring=(16, 3)):
    """2D overset workload modelled on the paper's 2D examples: the periodic
    box [0,2pi]^2 (n_box x n_box quads, session 0, interior nodes displaced
    by 0.05 h) overlapped by an annulus rho in [0.6, 1.4] around (pi, pi)
    (ring = (n_az, n_rad), session 1).  Queries: the boundary GLL nodes of
    each subdomain inside the other, tagged with their own session; fields
    u, v, p: the Walsh-type eddy u = -cos(x) sin(y), v = sin(x) cos(y),
    p = -(cos 2x + cos 2y)/4.  D^k in closed form."""
    lo, hi = (0.0, 0.0), (2 * np.pi, 2 * np.pi)
    cb = quad_mesh((n_box, n_box), N, lo=lo, hi=hi, amp_frac=0.05)
    c0 = (np.pi, np.pi)
    r_in, r_out = 0.6, 1.4
    cr, rho = ring_mesh(ring[0], ring[1], N, r_in, r_out, center=c0)
    db = rect_distance(cb, lo, hi)
    dr = np.maximum(np.minimum(rho - r_in, r_out - rho), 0.0)
    mesh = concat_meshes([cb, cr], N, [0, 1], [db, dr], name=f"walsh2d-N{N}")
    n = N + 1
    # annulus boundary nodes (inner and outer circles), deduplicated
    nodes = []
    for ea in range(ring[0]):
        for er, i in ((0, 0), (ring[1] - 1, N)):
            e = er + ring[1] * ea
            for j in range(N):                      # skip j = N (next element's j = 0)
                nodes.append(cr[:, e, i + n * j])
    qr = np.array(nodes).T
    # box nodes near the annulus: every box GLL node with r_in <= rho <= r_out (a volume set)
    xb = cb.reshape(2, -1)
    rb = np.hypot(xb[0] - c0[0], xb[1] - c0[1])
    keep = (rb > r_in) & (rb < r_out)
    qb = np.unique(np.round(xb[:, keep].T, 14), axis=0).T
    pts = np.ascontiguousarray(np.concatenate([qb, qr], axis=1))
    qsess = np.concatenate([np.zeros(qb.shape[1], np.int32), np.ones(qr.shape[1], np.int32)])
    X, Y = mesh.coords
    fields = np.stack([-np.cos(X) * np.sin(Y), np.sin(X) * np.cos(Y), -(np.cos(2 * X) + np.cos(2 * Y)) / 4])
    return mesh, Queries(pts=pts, qsess=qsess, fields=np.ascontiguousarray(fields),
                         info={"P_box": int(qb.shape[1]), "P_ring": int(qr.shape[1])})
