"""Seeded synthetic GelSight-style workloads: gel meshes, rigid indenter meshes, pose trajectories.

This module only BUILDS INPUTS.  It holds none of the solver's arithmetic (no energy, no
derivatives, no surface extraction, no masses): both the CUDA library and the CPU oracle receive
exactly the arrays produced here and derive everything else on their own.

Geometry follows the TacEx setting (the gelpad of a GelSight Mini pressed by a rigid object, the
"ball rolling" / pushing scenes of the paper's Sec. 3, GIPC step of Sec. "General GIPC Simulation
Pipeline"): a box-shaped gel whose bottom face is held fixed, and a kinematic rigid indenter that
moves along a prescribed pose trajectory.  The paper ships no meshes; these are stand-ins with the
stated sizes:

* gel: axis-aligned box meshed as an nx*ny*nz vertex grid, every cube split into the 6 Kuhn
  tetrahedra that share the cube's (0,0,0)-(1,1,1) diagonal (conforming across cubes);
* indenters: icosphere, capped cylinder lying with its axis parallel to the top face, and a
  triangular prism resting on one edge;
* trajectories: the indenter starts with its lowest point one barrier distance d_hat above the top
  face and is pressed to the nominal depth linearly in time (optionally followed by a tangential
  slide along +x).

All lengths are metres, poses are (qw, qx, qy, qz, tx, ty, tz).
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

IDENTITY_Q = (1.0, 0.0, 0.0, 0.0)

# Material and barrier settings shared by all GelSight workloads (gel: E = 0.3 MPa, nu = 0.45,
# rho = 1100 kg/m^3; barrier distance d_hat = 0.1 mm; time step 1/60 s).
YOUNG = 0.3e6
POISSON = 0.45
DENSITY = 1100.0
DHAT = 1.0e-4
DT = 1.0 / 60.0
NEWTON_TOL = 1.0e-5  # relative: ||p||_inf / h < NEWTON_TOL * (gel bounding-box diagonal)

# Grids used by the workloads: (vertex counts, box size in metres).
GRID_SMALL = ((10, 13, 4), (0.018, 0.024, 0.004))
GRID_MID = ((21, 26, 5), (0.020, 0.025, 0.004))
GRID_MINI = ((41, 51, 9), (0.020, 0.025, 0.004))


@dataclasses.dataclass
class GelMesh:
    verts: np.ndarray  # (N, 3) float64, rest positions
    tets: np.ndarray  # (T, 4) int32, positively oriented
    dirichlet: np.ndarray  # (N,) uint8, 1 = held at its rest position

    @property
    def top(self) -> float:
        return float(self.verts[:, 2].max())


@dataclasses.dataclass
class Indenter:
    verts: np.ndarray  # (M, 3) float64 in the indenter frame
    tris: np.ndarray  # (K, 3) int32
    kind: str


@dataclasses.dataclass
class Workload:
    name: str
    gel: GelMesh
    indenter: Indenter
    pose0: np.ndarray  # (7,)
    poses: np.ndarray  # (S, 7): target pose of step s (s = 0..S-1)
    dt: float
    material: tuple = (YOUNG, POISSON, DENSITY)
    dhat: float = DHAT
    newton_tol: float = NEWTON_TOL


# ----------------------------------------------------------------------------------------------
# gel
# ----------------------------------------------------------------------------------------------
def gel_grid(nx: int, ny: int, nz: int, size) -> GelMesh:
    """Box gel on an nx*ny*nz vertex grid, 6 Kuhn tets per cube, bottom face (z = 0) fixed."""
    verts, tets, dirichlet = _gel_grid_arrays(int(nx), int(ny), int(nz), tuple(float(v) for v in size))
    return GelMesh(verts.copy(), tets.copy(), dirichlet.copy())


@functools.lru_cache(maxsize=16)
def _gel_grid_arrays(nx, ny, nz, size):
    lx, ly, lz = size
    return _tensor_grid_arrays(np.linspace(0.0, lx, nx), np.linspace(0.0, ly, ny), np.linspace(0.0, lz, nz))


def _tensor_grid_arrays(xs, ys, zs):
    nx, ny, nz = len(xs), len(ys), len(zs)
    zz, yy, xx = np.meshgrid(zs, ys, xs, indexing="ij")
    verts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1).astype(np.float64)
    # cube origins (i, j, k), ordered k-major then j then i (x fastest)
    kk, jj, ii = np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    base = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
    axes = np.eye(3, dtype=np.int64)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]

    def vid(c):
        return c[:, 0] + nx * (c[:, 1] + ny * c[:, 2])

    per_cube = []
    for p in perms:
        c0 = base
        c1 = c0 + axes[p[0]]
        c2 = c1 + axes[p[1]]
        c3 = c2 + axes[p[2]]
        t = np.stack([vid(c0), vid(c1), vid(c2), vid(c3)], axis=1)
        # orientation of this path tet = sign of the axis permutation
        if np.linalg.det(np.stack([axes[p[0]], axes[p[1]], axes[p[2]]])) < 0:
            t = t[:, [0, 1, 3, 2]]
        per_cube.append(t)
    tets = np.stack(per_cube, axis=1).reshape(-1, 4).astype(np.int32)
    dirichlet = (verts[:, 2] <= 1e-12).astype(np.uint8)
    return verts, tets, dirichlet


def graded_axis(length: float, h0: float, ratio: float, centred: bool) -> np.ndarray:
    """Node coordinates on [0, length] with cell size h0 at the centre (centred) or at the top end
    (length), growing geometrically by `ratio` away from it; the outermost cell absorbs the rest."""
    half = 0.5 * length if centred else length
    cuts, x, h = [0.0], 0.0, h0
    while x + h < half - 0.5 * h:
        x += h
        cuts.append(x)
        h *= ratio
    cuts.append(half)
    c = np.asarray(cuts)
    if centred:
        return np.concatenate([half - c[::-1], half + c[1:]])
    return length - c[::-1]


def gel_tensor_grid(xs, ys, zs) -> GelMesh:
    """Box gel on the tensor-product grid xs x ys x zs (Kuhn tets, bottom face fixed)."""
    verts, tets, dirichlet = _tensor_grid_arrays(np.asarray(xs, float), np.asarray(ys, float), np.asarray(zs, float))
    return GelMesh(verts, tets, dirichlet)


# ----------------------------------------------------------------------------------------------
# indenters
# ----------------------------------------------------------------------------------------------
def spherical_cap(radius: float, cap_radius: float, n_rings: int, n_sectors: int, grading: float = 1.0) -> Indenter:
    """Lower cap of a sphere of `radius`, apex at the frame origin (centre at z = radius), out to
    the ring of horizontal radius cap_radius: an apex fan and n_rings rings of n_sectors vertices
    (ring spacing graded by `grading`, finest at the apex) -- an open triangle mesh."""
    th_max = math.asin(min(cap_radius / radius, 1.0))
    w = np.cumsum(grading ** np.arange(n_rings))
    th = th_max * w / w[-1]
    verts = [np.zeros(3)]
    for t in th:
        for k in range(n_sectors):
            ph = 2.0 * math.pi * (k + 0.5 * (len(verts) % 2)) / n_sectors
            verts.append(np.array([radius * math.sin(t) * math.cos(ph), radius * math.sin(t) * math.sin(ph),
                                   radius * (1.0 - math.cos(t))]))
    tris = []
    for k in range(n_sectors):
        tris.append((0, 1 + k, 1 + (k + 1) % n_sectors))
    for r in range(n_rings - 1):
        a0, b0 = 1 + r * n_sectors, 1 + (r + 1) * n_sectors
        for k in range(n_sectors):
            k1 = (k + 1) % n_sectors
            tris.append((a0 + k, b0 + k, b0 + k1))
            tris.append((a0 + k, b0 + k1, a0 + k1))
    return Indenter(np.array(verts), np.array(tris, dtype=np.int32), "cap")

def icosphere(radius: float, level: int) -> Indenter:
    """Icosahedron subdivided `level` times, vertices on the sphere (level 2: 162 verts, 320 tris)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
         (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return Indenter(np.asarray(verts) * radius, np.asarray(faces, dtype=np.int32), "sphere")


def cylinder(radius: float, length: float, n_around: int, n_along: int) -> Indenter:
    """Closed cylinder with its axis along y (parallel to the gel's top face), centred at 0."""
    verts, tris = [], []
    for a in range(n_along + 1):
        y = -0.5 * length + length * a / n_along
        for r in range(n_around):
            th = 2.0 * math.pi * (r + 0.5) / n_around
            verts.append((radius * math.sin(th), y, -radius * math.cos(th)))
    for a in range(n_along):
        for r in range(n_around):
            i0 = a * n_around + r
            i1 = a * n_around + (r + 1) % n_around
            j0, j1 = i0 + n_around, i1 + n_around
            tris += [(i0, j0, i1), (i1, j0, j1)]
    c0 = len(verts)
    verts.append((0.0, -0.5 * length, 0.0))
    c1 = len(verts)
    verts.append((0.0, 0.5 * length, 0.0))
    last = n_along * n_around
    for r in range(n_around):
        tris.append((c0, r, (r + 1) % n_around))
        tris.append((c1, last + (r + 1) % n_around, last + r))
    return Indenter(np.asarray(verts, dtype=np.float64), np.asarray(tris, dtype=np.int32), "cylinder")


def prism(side: float, length: float, n_along: int, n_side: int) -> Indenter:
    """Triangular prism (equilateral cross-section of edge `side`) lying on one edge; axis along y."""
    h = side * math.sqrt(3.0) / 2.0
    # cross-section corners in (x, z): the bottom edge-vertex, then the two top corners
    corners = [(0.0, -2.0 * h / 3.0), (0.5 * side, h / 3.0), (-0.5 * side, h / 3.0)]
    ring = []
    for c in range(3):
        p, q = corners[c], corners[(c + 1) % 3]
        for s in range(n_side):
            w = s / n_side
            ring.append((p[0] + w * (q[0] - p[0]), p[1] + w * (q[1] - p[1])))
    nr = len(ring)
    verts, tris = [], []
    for a in range(n_along + 1):
        y = -0.5 * length + length * a / n_along
        for (x, z) in ring:
            verts.append((x, y, z))
    for a in range(n_along):
        for r in range(nr):
            i0 = a * nr + r
            i1 = a * nr + (r + 1) % nr
            j0, j1 = i0 + nr, i1 + nr
            tris += [(i0, i1, j0), (i1, j1, j0)]
    # caps: fan around each cap's centroid
    for a, sign in ((0, -1), (n_along, 1)):
        y = -0.5 * length + length * a / n_along
        c = len(verts)
        verts.append((0.0, y, 0.0))
        for r in range(nr):
            i0 = a * nr + r
            i1 = a * nr + (r + 1) % nr
            tris.append((c, i1, i0) if sign < 0 else (c, i0, i1))
    return Indenter(np.asarray(verts, dtype=np.float64), np.asarray(tris, dtype=np.int32), "prism")


def indenter_by_tri_count(rng: np.random.Generator, kind: str, n_tri: int) -> Indenter:
    """Shapes of the GelSight-Mini workloads, realised with a triangle count close to `n_tri`."""
    if kind == "sphere":
        r = float(rng.uniform(0.002, 0.006))
        level = 2 if abs(n_tri - 320) <= abs(n_tri - 1280) else 3
        return icosphere(r, level)
    if kind == "cylinder":
        # tris = 2*na*nl + 2*na
        na = 24
        nl = max(1, int(round((n_tri - 2 * na) / (2 * na))))
        return cylinder(0.002, 0.010, na, nl)
    if kind == "prism":
        # tris = 2*3*ns*nl + 2*3*ns
        ns = 4
        nl = max(1, int(round((n_tri - 6 * ns) / (6 * ns))))
        return prism(0.004, 0.010, nl, ns)
    raise ValueError(kind)


# ----------------------------------------------------------------------------------------------
# trajectories
# ----------------------------------------------------------------------------------------------
def pose(t, q=IDENTITY_Q) -> np.ndarray:
    return np.array([q[0], q[1], q[2], q[3], t[0], t[1], t[2]], dtype=np.float64)


def press_slide_poses(ind: Indenter, gel: GelMesh, center_xy, depth: float, n_press: int,
                      slide: float = 0.0, n_slide: int = 0, dhat: float = DHAT):
    """Start with the lowest indenter point d_hat above the top face, press by depth + d_hat
    linearly over n_press steps, then slide by `slide` along +x over n_slide steps."""
    z0 = gel.top + dhat - float(ind.verts[:, 2].min())
    start = np.array([center_xy[0], center_xy[1], z0])
    travel = depth + dhat
    poses = []
    for s in range(1, n_press + 1):
        poses.append(pose(start - np.array([0.0, 0.0, travel * s / n_press])))
    bottom = start - np.array([0.0, 0.0, travel])
    for s in range(1, n_slide + 1):
        poses.append(pose(bottom + np.array([slide * s / n_slide, 0.0, 0.0])))
    return pose(start), np.asarray(poses)


def small_gel_sphere(seed: int = 0, n_steps: int = 30, depth: float = 0.6e-3) -> Workload:
    """18x24x4 mm gel on a 10x13x4 grid (520 verts, 1944 tets), icosphere r = 5 mm (320 tris)
    pressed 0.6 mm over 30 steps; the seed fixes the x-y offset, uniform in +-3 mm."""
    rng = np.random.default_rng(seed)
    (nx, ny, nz), size = GRID_SMALL
    gel = gel_grid(nx, ny, nz, size)
    ind = icosphere(0.005, 2)
    off = rng.uniform(-0.003, 0.003, size=2)
    c = (0.5 * size[0] + off[0], 0.5 * size[1] + off[1])
    p0, poses = press_slide_poses(ind, gel, c, depth, n_steps)
    return Workload("gel10x13x4_sphere_r5mm_press0.6mm", gel, ind, p0, poses, DT)


def mini_gel(seed: int = 0, grid=GRID_MINI, depth: float = 1.0e-3, n_press: int = 60,
             slide: float = 2.0e-3, n_slide: int = 60, kind: str | None = None) -> Workload:
    """GelSight-Mini-scale gel (20x25x4 mm on a 41x51x9 grid: 18819 verts, 96000 tets) with a
    seeded indenter: sphere r in [2,6] mm, cylinder r 2 mm x 10 mm, or triangular prism of side
    4 mm (300-2000 tris); pressed 1.0 mm over 60 steps then slid 2 mm along +x over 60 steps."""
    rng = np.random.default_rng(seed)
    (nx, ny, nz), size = grid
    gel = gel_grid(nx, ny, nz, size)
    if kind is None:
        kind = ["sphere", "cylinder", "prism"][int(rng.integers(0, 3))]
    n_tri = int(rng.integers(300, 2001))
    ind = indenter_by_tri_count(rng, kind, n_tri)
    off = rng.uniform(-0.002, 0.002, size=2)
    c = (0.5 * size[0] + off[0] - 0.5 * slide, 0.5 * size[1] + off[1])
    p0, poses = press_slide_poses(ind, gel, c, depth, n_press, slide, n_slide)
    name = f"gel{nx}x{ny}x{nz}_{kind}{len(ind.tris)}_press{depth*1e3:.1f}mm_slide{slide*1e3:.1f}mm"
    return Workload(name, gel, ind, p0, poses, DT)


def hertz_block(h0: float = 0.06e-3, ratio: float = 1.3, half: float = 3.0e-3, thick: float = 2.0e-3,
                radius: float = 3.0e-3, depth: float = 40e-6, dhat: float = 5e-6, step: float = 4e-6,
                n_rings: int = 24, n_sectors: int = 48) -> Workload:
    """Hertz indentation: a 2*half x 2*half x thick block (bottom fixed, the gel material) meshed
    with cells of size h0 at the top centre growing by `ratio` outward and downward, pressed by
    a rigid spherical cap of `radius` to `depth` below the top face in quasi-static steps of
    `step` (time step 1 s, so inertia is negligible), barrier distance dhat."""
    xs = graded_axis(2 * half, h0, ratio, True)
    zs = graded_axis(thick, h0, ratio, False)
    gel = gel_tensor_grid(xs, xs, zs)
    a = math.sqrt(radius * depth)
    ind = spherical_cap(radius, min(3.0 * a, 0.9 * radius), n_rings, n_sectors, grading=1.08)
    n = int(math.ceil((depth + dhat) / step))
    p0, poses = press_slide_poses(ind, gel, (half, half), depth, n, dhat=dhat)
    return Workload(f"hertz_R{radius*1e3:.1f}mm_d{depth*1e6:.0f}um_h{h0*1e6:.0f}um", gel, ind, p0, poses, 1.0,
                    dhat=dhat)


def ball_mesh(n: int, radius: float, center) -> GelMesh:
    """Soft ball: an n*n*n vertex grid over the cube [-1, 1]^3 (6 Kuhn tets per cube) carried onto
    the ball by the concentric map p -> p |p|_inf / |p|_2 (the cube's faces onto the sphere), scaled
    by `radius` and moved to `center`; no vertex held.  n = 10, 20, 23 give 1000, 8000, 12167
    vertices and 4374, 41154, 63888 tets, next to the three soft-ball resolutions of Table 3."""
    verts, tets, _ = _tensor_grid_arrays(*(np.linspace(-1.0, 1.0, int(n)),) * 3)
    inf = np.abs(verts).max(axis=1)
    two = np.linalg.norm(verts, axis=1)
    scale = np.divide(inf, two, out=np.zeros_like(inf), where=two > 0)
    verts = verts * scale[:, None] * float(radius) + np.asarray(center, dtype=np.float64)
    e1, e2, e3 = (verts[tets[:, k]] - verts[tets[:, 0]] for k in (1, 2, 3))
    vol = np.einsum("ij,ij->i", np.cross(e1, e2), e3) / 6.0
    assert vol.min() > 0.0, "ball map inverted a tet"
    return GelMesh(verts, tets.astype(np.int32), np.zeros(len(verts), dtype=np.uint8))


def flat_plate(side: float, n: int) -> Indenter:
    """Square plate of `side` in the indenter frame's z = 0 plane (facing down), an n*n vertex grid,
    two triangles per cell."""
    t = np.linspace(-0.5 * side, 0.5 * side, n)
    yy, xx = np.meshgrid(t, t, indexing="ij")
    verts = np.stack([xx.ravel(), yy.ravel(), np.zeros(n * n)], axis=1)
    j, i = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    a = (i + n * j).ravel()
    tris = np.concatenate([np.stack([a, a + n, a + 1], 1), np.stack([a + 1, a + n, a + n + 1], 1)])
    return Indenter(verts, tris.astype(np.int32), "plate")


def join_meshes(a: GelMesh, b: GelMesh) -> GelMesh:
    """One tet mesh holding both bodies (b's vertices after a's): two connected components."""
    return GelMesh(np.concatenate([a.verts, b.verts]), np.concatenate([a.tets, b.tets + len(a.verts)]).astype(np.int32),
                   np.concatenate([a.dirichlet, b.dirichlet]))


def gel_ball(ball_n: int = 20, grid=GRID_MINI, radius: float = 4.0e-3, depth: float = 1.0e-3, n_press: int = 60,
             slide: float = 2.0e-3, n_slide: int = 60, seed: int = 0, gap_below: float = 2 * DHAT,
             gap_above: float = DHAT) -> Workload:
    """Soft ball between the gel and a rigid plate (the soft-ball scene of Table 3, the ball a
    deformable body of the gel's material): the ball (`ball_mesh`) rests gap_below above the gel's
    top face, its centre offset by a seeded +-1 mm in x-y; a 12 mm plate (`flat_plate`) starts
    gap_above above the ball, closes both gaps and squeezes `depth` over n_press steps, then slides
    along +x (without friction: over the ball).  Gaps below d_hat put both contacts in place from
    the first step."""
    rng = np.random.default_rng(seed)
    (nx, ny, nz), size = grid
    gel = gel_grid(nx, ny, nz, size)
    off = rng.uniform(-0.001, 0.001, size=2)
    c = np.array([0.5 * size[0] + off[0], 0.5 * size[1] + off[1], gel.top + gap_below + radius])
    ball = ball_mesh(ball_n, radius, c)
    ind = flat_plate(0.012, 13)
    start = np.array([c[0], c[1], float(ball.verts[:, 2].max()) + gap_above])
    travel = gap_below + gap_above + depth
    poses = [pose(start - np.array([0.0, 0.0, travel * s / n_press])) for s in range(1, n_press + 1)]
    bottom = start - np.array([0.0, 0.0, travel])
    poses += [pose(bottom + np.array([slide * s / n_slide, 0.0, 0.0])) for s in range(1, n_slide + 1)]
    name = f"gel{nx}x{ny}x{nz}_softball{len(ball.verts)}v_r{radius*1e3:.1f}mm_plate_press{depth*1e3:.1f}mm"
    return Workload(name, join_meshes(gel, ball), ind, pose(start), np.asarray(poses), DT)


def mixed_batch(n_gels: int = 256, seed0: int = 0, n_press: int = 60, n_slide: int = 60):
    """Batch of gels with resolutions drawn uniformly from the three grids, each with its own
    seeded indenter, trajectory and depth uniform in [0.2, 1.2] mm."""
    grids = [GRID_SMALL, GRID_MID, GRID_MINI]
    out = []
    for g in range(n_gels):
        rng = np.random.default_rng(10_000 + seed0 + g)
        grid = grids[int(rng.integers(0, 3))]
        depth = float(rng.uniform(0.2e-3, 1.2e-3))
        out.append(mini_gel(seed=seed0 + g, grid=grid, depth=depth, n_press=n_press,
                            slide=2.0e-3 if n_slide else 0.0, n_slide=n_slide))
    return out


def quat_mul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return (aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
            aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw)


def quat_axis_angle(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    s = math.sin(0.5 * angle)
    return (math.cos(0.5 * angle), axis[0] * s, axis[1] * s, axis[2] * s)
