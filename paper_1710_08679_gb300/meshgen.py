"""Seeded synthetic inputs: crust-shaped TET10 meshes, boundary masks and load cases.

This module only *describes* problems (geometry, connectivity, materials, boundary
masks, point forces, slip fields, observation points). It contains none of the
solver's arithmetic: no element stiffness, no assembly, no products. Both the
CUDA path and the CPU oracle consume what it produces.

Mesh recipe (the paper's crust models are not available, these stand in for them,
Sec. 4 and Sec. 5 describe layered crust blocks with a dipping plate interface):

* a box of nx*ny*nz hexahedra of edge h, each split into 6 tetrahedra along its
  (0,0,0)-(1,1,1) diagonal (one tetrahedron per permutation of the axes), which is
  conforming across hexahedra;
* second-order (10-node) tetrahedra in VTK order: corners 0..3, then the edge
  midpoints of (0,1), (1,2), (2,0), (0,3), (1,3), (2,3); every node lies on the
  (2nx+1)x(2ny+1)x(2nz+1) half-spacing lattice, the node id is the lattice index
  i + (2nx+1)*(j + (2ny+1)*k);
* interior vertex nodes (all-even lattice index, not on a face) are moved by
  U(-jitter*h, +jitter*h) per coordinate (numpy PCG64); boundary nodes are not moved
  so the faces stay planar; edge nodes are the exact midpoints of their edge, so
  every element is straight-sided (affine);
* vertex coordinates are snapped to a power-of-two grid fine enough that vertices,
  midpoints and vertex differences are all exact in FP32 (so FP64 and FP32 paths
  see the same geometry);
* z = 0 is the bottom (clamped), z = Lz the free surface, the x faces carry
  u_x = 0 and the y faces u_y = 0 (roller sides).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# VTK TET10 edge list: local edge node 4+q joins corners EDGES[q]
EDGES = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))

# the six axis permutations of the Kuhn split, with their parity
_PERMS = ((0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (1, 0, 2), (2, 1, 0))
_PARITY = (1, 1, 1, -1, -1, -1)


@dataclasses.dataclass
class Mesh:
    """A TET10 mesh plus its boundary mask.

    coords   float64 [N, 3]  (m)
    conn     int32   [E, 10] (0-based, VTK order)
    young    float64 [E]     (Pa)
    poisson  float64 [E]
    free     uint8   [N, 3]  1 = free DOF, 0 = Dirichlet (u = 0)
    """
    coords: np.ndarray
    conn: np.ndarray
    young: np.ndarray
    poisson: np.ndarray
    free: np.ndarray
    shape: Tuple[int, int, int]
    h: Tuple[float, float, float]
    lengths: Tuple[float, float, float]
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.conn.shape[0])

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes

    def lattice_shape(self) -> Tuple[int, int, int]:
        nx, ny, nz = self.shape
        return (2 * nx + 1, 2 * ny + 1, 2 * nz + 1)

    def node_id(self, i, j, k):
        """Node id of half-spacing lattice point (i, j, k)."""
        lx, ly, _ = self.lattice_shape()
        return np.asarray(i) + lx * (np.asarray(j) + ly * np.asarray(k))

    def centroids(self) -> np.ndarray:
        return self.coords[self.conn[:, :4]].mean(axis=1)


def _snap_quantum(max_abs: float) -> float:
    """Grid spacing 2^(e-23) with 2^e > max_abs: vertices on this grid have exactly
    representable FP32 midpoints and differences."""
    e = math.ceil(math.log2(max(max_abs, 1.0) * (1 + 1e-12)))
    return 2.0 ** (e - 23)


def box_mesh(shape: Tuple[int, int, int], lengths: Tuple[float, float, float],
             jitter: float = 0.0, seed: int = 0, name: str = "") -> Mesh:
    """Lattice TET10 mesh of the box [0,Lx]x[0,Ly]x[0,Lz]; materials are filled with
    a placeholder (set them with one of the layer functions)."""
    nx, ny, nz = (int(s) for s in shape)
    Lx, Ly, Lz = (float(v) for v in lengths)
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    lx, ly, lz = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    N = lx * ly * lz
    ii, jj, kk = np.meshgrid(np.arange(lx), np.arange(ly), np.arange(lz), indexing="ij")
    # node id order: i fastest, then j, then k
    ii = ii.transpose(2, 1, 0).reshape(-1)
    jj = jj.transpose(2, 1, 0).reshape(-1)
    kk = kk.transpose(2, 1, 0).reshape(-1)
    coords = np.stack([ii * (hx / 2), jj * (hy / 2), kk * (hz / 2)], axis=1).astype(np.float64)

    vertex = (ii % 2 == 0) & (jj % 2 == 0) & (kk % 2 == 0)
    interior = (ii > 0) & (ii < lx - 1) & (jj > 0) & (jj < ly - 1) & (kk > 0) & (kk < lz - 1)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        move = vertex & interior
        nm = int(move.sum())
        d = rng.uniform(-1.0, 1.0, size=(nm, 3)) * (jitter * np.array([hx, hy, hz]))
        coords[move] += d
    q = _snap_quantum(max(Lx, Ly, Lz))
    coords[vertex] = np.round(coords[vertex] / q) * q
    # boundary planes stay exact (the lattice values there may not be on the grid)
    coords[ii == 0, 0] = 0.0
    coords[ii == lx - 1, 0] = Lx
    coords[jj == 0, 1] = 0.0
    coords[jj == ly - 1, 1] = Ly
    coords[kk == 0, 2] = 0.0
    coords[kk == lz - 1, 2] = Lz
    # edge (non-vertex) nodes: exact midpoint of the Kuhn edge through them, which
    # joins lattice points p - d and p + d with d = (i%2, j%2, k%2)
    nv = ~vertex
    di, dj, dk = ii[nv] % 2, jj[nv] % 2, kk[nv] % 2
    a = (ii[nv] - di) + lx * ((jj[nv] - dj) + ly * (kk[nv] - dk))
    b = (ii[nv] + di) + lx * ((jj[nv] + dj) + ly * (kk[nv] + dk))
    coords[nv] = 0.5 * (coords[a] + coords[b])

    # connectivity, hexahedra in (k, j, i) order, 6 tetrahedra each
    hi, hj, hk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hi = hi.transpose(2, 1, 0).reshape(-1)
    hj = hj.transpose(2, 1, 0).reshape(-1)
    hk = hk.transpose(2, 1, 0).reshape(-1)
    nh = hi.size
    base = np.stack([2 * hi, 2 * hj, 2 * hk], axis=1)  # [nh, 3] lattice coords
    conn = np.empty((nh, 6, 10), dtype=np.int64)
    eye = np.eye(3, dtype=np.int64) * 2
    for t, (perm, par) in enumerate(zip(_PERMS, _PARITY)):
        p0 = base
        p1 = base + eye[perm[0]]
        p2 = p1 + eye[perm[1]]
        p3 = base + 2
        if par < 0:
            p1, p2 = p2, p1
        corners = (p0, p1, p2, p3)
        pts = list(corners) + [(corners[a] + corners[b]) // 2 for a, b in EDGES]
        for ln, p in enumerate(pts):
            conn[:, t, ln] = p[:, 0] + lx * (p[:, 1] + ly * p[:, 2])
    conn = conn.reshape(-1, 10).astype(np.int32)

    free = np.ones((N, 3), dtype=np.uint8)
    free[kk == 0, :] = 0
    free[(ii == 0) | (ii == lx - 1), 0] = 0
    free[(jj == 0) | (jj == ly - 1), 1] = 0
    E = conn.shape[0]
    return Mesh(coords=coords, conn=conn, young=np.full(E, 1.0e10), poisson=np.full(E, 0.25),
                free=free, shape=(nx, ny, nz), h=(hx, hy, hz), lengths=(Lx, Ly, Lz), name=name)


# ---------------------------------------------------------------------------
# layered crust with a dipping interface
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Interface:
    """Plane striking along y, dipping `dip_deg` toward +x, reaching the surface
    z = z_top at x = x0. Points with depth below the plane's depth at their x are
    in the footwall; above it, in the hanging wall."""
    x0: float
    z_top: float
    dip_deg: float

    def depth_of_plane(self, x):
        return (np.asarray(x) - self.x0) * math.tan(math.radians(self.dip_deg))

    def hanging_wall(self, pts: np.ndarray) -> np.ndarray:
        depth = self.z_top - pts[:, 2]
        return depth < self.depth_of_plane(pts[:, 0])

    def plane_coords(self, pts: np.ndarray) -> np.ndarray:
        """(along-strike y, down-dip distance, signed normal distance) of points."""
        s, c = math.sin(math.radians(self.dip_deg)), math.cos(math.radians(self.dip_deg))
        dx = pts[:, 0] - self.x0
        dd = self.z_top - pts[:, 2]  # depth
        down_dip = dx * c + dd * s
        normal = dx * s - dd * c      # > 0 : hanging-wall side
        return np.stack([pts[:, 1], down_dip, normal], axis=1)

    def dip_vector(self) -> np.ndarray:
        s, c = math.sin(math.radians(self.dip_deg)), math.cos(math.radians(self.dip_deg))
        return np.array([c, 0.0, -s])

    def strike_vector(self) -> np.ndarray:
        return np.array([0.0, 1.0, 0.0])


def set_two_layers(mesh: Mesh, z_split: float, upper=(40e9, 0.25), lower=(80e9, 0.27)) -> None:
    zc = mesh.centroids()[:, 2]
    up = zc > z_split
    mesh.young = np.where(up, upper[0], lower[0]).astype(np.float64)
    mesh.poisson = np.where(up, upper[1], lower[1]).astype(np.float64)


def set_dipping_layers(mesh: Mesh, iface: Interface, depths: List[float],
                       materials: List[Tuple[float, float]], offset: float) -> None:
    """Layer boundaries at the given depths below the surface; on the hanging-wall
    side every boundary is shallower by `offset` (a fault throw across the plane)."""
    assert len(materials) == len(depths) + 1
    cen = mesh.centroids()
    depth = iface.z_top - cen[:, 2]
    hw = iface.hanging_wall(cen)
    eff = depth + np.where(hw, offset, 0.0)
    layer = np.searchsorted(np.asarray(depths, dtype=np.float64), eff, side="right")
    mat = np.asarray(materials, dtype=np.float64)
    mesh.young = mat[layer, 0].copy()
    mesh.poisson = mat[layer, 1].copy()


# ---------------------------------------------------------------------------
# load cases
# ---------------------------------------------------------------------------

def double_couple(mesh: Mesh, center_lattice: Tuple[int, int, int], force: float) -> np.ndarray:
    """Strike-slip (M_xy) double couple: +F x at centre+s*y, -F x at centre-s*y,
    +F y at centre+s*x, -F y at centre-s*x; s = one half-spacing lattice step.
    Returns f [N, 3]."""
    i, j, k = center_lattice
    f = np.zeros((mesh.n_nodes, 3))
    f[mesh.node_id(i, j + 1, k), 0] += force
    f[mesh.node_id(i, j - 1, k), 0] -= force
    f[mesh.node_id(i + 1, j, k), 1] += force
    f[mesh.node_id(i - 1, j, k), 1] -= force
    return f * mesh.free


@dataclasses.dataclass
class SlipCase:
    """Unit slip on a fault patch, to be turned into split-node forces by the
    solver side: f = -sum over `elems` of K_e s_e (then masked). `slip` is the
    nodal slip field [N, 3] (nonzero only on interface nodes of the patch)."""
    elems: np.ndarray      # int64 [m] hanging-wall elements touching the patch nodes
    slip: np.ndarray       # float64 [N, 3]
    center: Tuple[float, float]
    size: float
    direction: str


def interface_nodes(mesh: Mesh, iface: Interface) -> Tuple[np.ndarray, np.ndarray]:
    """Nodes shared by hanging-wall and footwall elements (the discrete fault surface
    made of element faces), and the hanging-wall element mask."""
    hw = iface.hanging_wall(mesh.centroids())
    N = mesh.n_nodes
    in_hw = np.zeros(N, dtype=bool)
    in_fw = np.zeros(N, dtype=bool)
    in_hw[mesh.conn[hw].reshape(-1)] = True
    in_fw[mesh.conn[~hw].reshape(-1)] = True
    on = in_hw & in_fw
    # the box faces are not part of the fault
    return on, hw


def bspline3(t: np.ndarray) -> np.ndarray:
    """Centred cubic B-spline of unit knot spacing (support [-2, 2], B(0) = 2/3)."""
    a = np.abs(np.asarray(t, dtype=np.float64))
    return np.where(a < 1.0, 2.0 / 3.0 - a * a + 0.5 * a ** 3,
                    np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))


def slip_patch(mesh: Mesh, iface: Interface, on_iface: np.ndarray, hw: np.ndarray,
               center: Tuple[float, float], size: float, direction: str,
               profile: str = "uniform") -> SlipCase:
    """Unit slip on the interface nodes within a size x size patch (fault-plane
    coordinates). profile "uniform": slip 1 on the whole patch; "bspline": slip
    B(4 s / size) B(4 d / size) / B(0)^2 in the along-strike and down-dip offsets
    (s, d) from the centre, a tensor cubic B-spline that is 1 at the centre and
    vanishes smoothly at the patch edge (the paper's unit B-spline slips, Sec. 5)."""
    pc = iface.plane_coords(mesh.coords)
    half = 0.5 * size
    sel = on_iface & (np.abs(pc[:, 0] - center[0]) <= half + 1e-9) & \
        (np.abs(pc[:, 1] - center[1]) <= half + 1e-9)
    vec = iface.dip_vector() if direction == "dip" else iface.strike_vector()
    slip = np.zeros((mesh.n_nodes, 3))
    if profile == "uniform":
        slip[sel] = vec
    elif profile == "bspline":
        amp = bspline3(4.0 * (pc[sel, 0] - center[0]) / size) * bspline3(4.0 * (pc[sel, 1] - center[1]) / size)
        amp /= (2.0 / 3.0) ** 2
        slip[sel] = amp[:, None] * vec[None, :]
        sel = sel.copy()
        sel[np.nonzero(sel)[0][amp == 0.0]] = False
    else:
        raise ValueError(f"unknown slip profile {profile!r}")
    touch = np.zeros(mesh.n_elem, dtype=bool)
    touch |= np.any(sel[mesh.conn], axis=1)
    elems = np.nonzero(touch & hw)[0]
    return SlipCase(elems=elems, slip=slip, center=center, size=size, direction=direction)


# ---------------------------------------------------------------------------
# observation points on the free surface (adjoint workload)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Observations:
    """u_obs[p, c] = sum_a weight[p, a] * u[node[p, a], c] for the 6-node quadratic
    triangle of the top-face TET10 face containing point p."""
    points: np.ndarray   # [P, 2] (x, y)
    node: np.ndarray     # int64 [P, 6]
    weight: np.ndarray   # float64 [P, 6]

    def matrix(self, n_nodes: int):
        """Sparse [3P, 3N] observation operator (scipy CSR), row 3p+c."""
        import scipy.sparse as sp
        P = self.node.shape[0]
        rows = (3 * np.arange(P)[:, None, None] + np.arange(3)[None, None, :]) * np.ones((1, 6, 1), np.int64)
        cols = 3 * self.node[:, :, None] + np.arange(3)[None, None, :]
        vals = np.repeat(self.weight[:, :, None], 3, axis=2)
        return sp.csr_matrix((vals.reshape(-1), (rows.reshape(-1), cols.reshape(-1))),
                             shape=(3 * P, 3 * n_nodes))


def surface_observations(mesh: Mesh, n_points: int, xy_range: Tuple[float, float], seed: int) -> Observations:
    """Uniform random points on the top face. The top face is an unjittered lattice
    whose squares are split along the (0,0)-(1,1) diagonal by the hexahedron split."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.uniform(xy_range[0], xy_range[1], size=(n_points, 2))
    nx, ny, nz = mesh.shape
    hx, hy, _ = mesh.h
    ci = np.minimum((pts[:, 0] // hx).astype(np.int64), nx - 1)
    cj = np.minimum((pts[:, 1] // hy).astype(np.int64), ny - 1)
    xi = pts[:, 0] / hx - ci
    eta = pts[:, 1] / hy - cj
    ktop = 2 * nz
    # triangle A: (0,0),(1,0),(1,1) when xi >= eta ; B: (0,0),(0,1),(1,1)
    a = xi >= eta
    # barycentric coordinates on the unit square triangles
    L = np.empty((n_points, 3))
    c1 = np.where(a[:, None], np.array([1, 0])[None, :], np.array([0, 1])[None, :])
    # corners in lattice units (half steps): v0=(0,0), v1=(2,0) or (0,2), v2=(2,2)
    L[:, 0] = 1.0 - np.maximum(xi, eta)
    L[:, 1] = np.abs(xi - eta)
    L[:, 2] = np.minimum(xi, eta)
    v = np.zeros((n_points, 3, 2), dtype=np.int64)
    v[:, 1, :] = 2 * c1
    v[:, 2, :] = 2
    bi, bj = 2 * ci, 2 * cj
    tri_nodes = []
    for (p, q) in ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)):
        li = bi + (v[:, p, 0] + v[:, q, 0]) // 2
        lj = bj + (v[:, p, 1] + v[:, q, 1]) // 2
        tri_nodes.append(mesh.node_id(li, lj, ktop))
    node = np.stack(tri_nodes, axis=1).astype(np.int64)
    # barycentric coordinates from the actual (grid-snapped) corner positions
    P0 = mesh.coords[node[:, 0], :2]
    P1 = mesh.coords[node[:, 1], :2]
    P2 = mesh.coords[node[:, 2], :2]
    A = np.stack([P1 - P0, P2 - P0], axis=2)            # [P, 2, 2]
    l12 = np.linalg.solve(A, (pts - P0)[:, :, None])[:, :, 0]
    L[:, 1] = l12[:, 0]
    L[:, 2] = l12[:, 1]
    L[:, 0] = 1.0 - L[:, 1] - L[:, 2]
    w = np.empty((n_points, 6))
    w[:, 0] = L[:, 0] * (2 * L[:, 0] - 1)
    w[:, 1] = L[:, 1] * (2 * L[:, 1] - 1)
    w[:, 2] = L[:, 2] * (2 * L[:, 2] - 1)
    w[:, 3] = 4 * L[:, 0] * L[:, 1]
    w[:, 4] = 4 * L[:, 1] * L[:, 2]
    w[:, 5] = 4 * L[:, 0] * L[:, 2]
    return Observations(points=pts, node=node, weight=w)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def plain_box(seed: int = 0, jitter: float = 0.10, n: int = 8) -> Mesh:
    """8 km box, n^3 hexahedra, two horizontal layers split at z = 4 km:
    (40 GPa, 0.25) above, (80 GPa, 0.27) below."""
    m = box_mesh((n, n, n), (8000.0, 8000.0, 8000.0), jitter=jitter, seed=seed,
                 name=f"box8km_{n}^3")
    set_two_layers(m, 4000.0)
    return m


def plain_box_rhs(mesh: Mesh, force: float = 1.0e12) -> np.ndarray:
    """Double couple of magnitude `force` at the box centre; f [N, 1, 3]."""
    lx, ly, lz = mesh.lattice_shape()
    return double_couple(mesh, (lx // 2, ly // 2, lz // 2), force)[:, None, :]


CRUST4 = [(1.0e10, 0.30), (4.0e10, 0.27), (8.0e10, 0.25), (1.2e11, 0.22)]


def crust_interface(lengths) -> Interface:
    Lx, Ly, Lz = lengths
    return Interface(x0=Lx / 14.0, z_top=Lz, dip_deg=30.0)


def crust_block(shape=(70, 70, 35), h: float = 1000.0, jitter: float = 0.15, seed: int = 1,
                n_layers: int = 4) -> Tuple[Mesh, Interface]:
    """Layered crust block of 1 km hexahedra with a 30-degree dipping interface;
    layer boundaries offset 2 km across the interface."""
    lengths = tuple(float(s) * h for s in shape)
    m = box_mesh(shape, lengths, jitter=jitter, seed=seed,
                 name=f"crust_{shape[0]}x{shape[1]}x{shape[2]}")
    iface = crust_interface(lengths)
    Lz = lengths[2]
    if n_layers == 4:
        mats = CRUST4
    else:
        E = np.geomspace(1.0e10, 1.2e11, n_layers)
        nu = np.linspace(0.30, 0.22, n_layers)
        mats = list(zip(E.tolist(), nu.tolist()))
    depths = [Lz * (i + 1) / (n_layers + 1) for i in range(n_layers - 1)]
    set_dipping_layers(m, iface, depths, mats, offset=2000.0)
    return m, iface


# The paper's two-layer measurement model (its table of material properties):
# (Vp m/s, Vs m/s, density kg/m^3) of layer 1 (top) and layer 2.
PAPER_LAYERS = ((1600.0, 400.0, 1850.0), (5800.0, 3000.0, 2700.0))


def elastic_from_velocities(vp: float, vs: float, rho: float) -> Tuple[float, float]:
    """Isotropic (E, nu) of a medium with P and S wave speeds vp, vs and density
    rho: mu = rho vs^2, lambda = rho (vp^2 - 2 vs^2)."""
    mu = rho * vs * vs
    lam = rho * (vp * vp - 2.0 * vs * vs)
    return mu * (3.0 * lam + 2.0 * mu) / (lam + mu), lam / (2.0 * (lam + mu))


def two_layer_block(shape=(70, 70, 35), h: float = 1000.0, soft_thickness: float = 5000.0,
                    jitter: float = 0.15, seed: int = 4) -> Tuple[Mesh, Interface]:
    """The paper's two-layer model on a crust block: layer 1 (Vp 1,600 m/s, Vs 400
    m/s, 1,850 kg/m^3: E = 0.87 GPa, nu = 0.467) in the top `soft_thickness`, layer
    2 (5,800 / 3,000 / 2,700: E = 64 GPa, nu = 0.317) below, split by element
    centroid; the dipping interface of the crust blocks carries the slip sources."""
    lengths = tuple(float(v) * h for v in shape)
    m = box_mesh(shape, lengths, jitter=jitter, seed=seed, name=f"two_layer_{shape[0]}x{shape[1]}x{shape[2]}")
    iface = crust_interface(lengths)
    set_two_layers(m, lengths[2] - soft_thickness, upper=elastic_from_velocities(*PAPER_LAYERS[0]),
                   lower=elastic_from_velocities(*PAPER_LAYERS[1]))
    return m, iface


def random_vectors(n_nodes: int, R: int, seed: int) -> np.ndarray:
    """x ~ N(0,1), float64 [N, R, 3] (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n_nodes, R, 3))


def patch_grid_cases(mesh: Mesh, iface: Interface, n_along: int = 4, spacing: float = 4000.0,
                     size: float = 2000.0, direction: str = "dip", profile: str = "uniform") -> List[SlipCase]:
    """n_along x n_along patches centred in the box, `spacing` apart along strike
    and along dip."""
    on, hw = interface_nodes(mesh, iface)
    Lx, Ly, Lz = mesh.lengths
    dip_len = Lz / math.sin(math.radians(iface.dip_deg))
    # stay inside the box: the down-dip extent reaching x = Lx
    x_end = min(Lx, iface.x0 + Lz / math.tan(math.radians(iface.dip_deg)))
    dd_end = (x_end - iface.x0) / math.cos(math.radians(iface.dip_deg))
    mid_dd = 0.5 * min(dip_len, dd_end)
    mid_y = 0.5 * Ly
    offs = (np.arange(n_along) - 0.5 * (n_along - 1)) * spacing
    cases = []
    for a in offs:
        for b in offs:
            cases.append(slip_patch(mesh, iface, on, hw, (mid_y + a, mid_dd + b), size, direction, profile))
    return cases


def many_cases(mesh: Mesh, iface: Interface, n_patches: int = 48, seed: int = 3) -> List[SlipCase]:
    """n_patches random patches (1-4 km, random depth) x 2 slip directions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    on, hw = interface_nodes(mesh, iface)
    Lx, Ly, Lz = mesh.lengths
    x_end = min(Lx, iface.x0 + Lz / math.tan(math.radians(iface.dip_deg)))
    dd_end = (x_end - iface.x0) / math.cos(math.radians(iface.dip_deg))
    cases = []
    for _ in range(n_patches):
        size = float(rng.uniform(1000.0, 4000.0))
        y = float(rng.uniform(0.2 * Ly, 0.8 * Ly))
        dd = float(rng.uniform(0.1 * dd_end + size, 0.9 * dd_end - size))
        for d in ("strike", "dip"):
            cases.append(slip_patch(mesh, iface, on, hw, (y, dd), size, d))
    return cases


def adjoint_box(n: int = 24, seed: int = 0, jitter: float = 0.10) -> Mesh:
    return plain_box(seed=seed, jitter=jitter, n=n)


def adjoint_sources(mesh: Mesh, force: float = 1.0e12) -> np.ndarray:
    """16 unit double couples at (x, y) in {1,3,5,7} km, z = 4 km on the 8 km box;
    f [N, 16, 3]. Requires the lattice to have a node at those points."""
    lx, ly, lz = mesh.lattice_shape()
    Lx, Ly, Lz = mesh.lengths
    out = np.zeros((mesh.n_nodes, 16, 3))
    r = 0
    for xs in (1000.0, 3000.0, 5000.0, 7000.0):
        for ys in (1000.0, 3000.0, 5000.0, 7000.0):
            i = int(round(xs / Lx * (lx - 1)))
            j = int(round(ys / Ly * (ly - 1)))
            k = int(round(4000.0 / Lz * (lz - 1)))
            out[:, r, :] = double_couple(mesh, (i, j, k), force)
            r += 1
    return out


def adjoint_true_logE(mesh: Mesh) -> np.ndarray:
    """m_true = log E + 0.2 exp(-|x - (4,4,6) km|^2 / (2 (1.5 km)^2)) per element."""
    c = mesh.centroids()
    d2 = np.sum((c - np.array([4000.0, 4000.0, 6000.0])) ** 2, axis=1)
    return np.log(mesh.young) + 0.2 * np.exp(-d2 / (2 * 1500.0 ** 2))


def noise(shape, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape)


def unit_directions(n_dir: int, n_params: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((n_dir, n_params))
    return v / np.linalg.norm(v, axis=1, keepdims=True)
