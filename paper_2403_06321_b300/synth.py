"""Seeded synthetic inputs: Kuhn-split cube-grid tetrahedral meshes and states.

This module only produces inputs (topology, rest positions, materials, pins,
initial states).  It contains none of the method's arithmetic: no rest-shape
matrices, masses, energies or solves.  Both the CUDA path and the CPU oracle
are fed from here, and neither of them is imported by it.

The paper's meshes (armadillo, squishy balls, teapot, ...) are not available,
so regular grids of cubes, each split into 6 tetrahedra, stand in for them
(Sec. 5 scenes are volumetric tet meshes with 6-9 vertex colours).
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Optional

import numpy as np

FACES = ("x-", "x+", "y-", "y+", "z-", "z+")


@dataclasses.dataclass
class MeshInput:
    """One tetrahedral mesh in the caller's vertex order."""

    rest: np.ndarray  # (N, 3) float64 rest positions
    tets: np.ndarray  # (T, 4) int32 vertex ids
    young: np.ndarray  # (T,) float32 Young's modulus [Pa]
    poisson: np.ndarray  # (T,) float32 Poisson ratio
    density: np.ndarray  # (T,) float32 [kg/m^3]
    pinned: np.ndarray  # (N,) uint8, 1 = position fixed (bilateral constraint)
    grid_ijk: Optional[np.ndarray] = None  # (N, 3) int32 lattice coordinates
    # subspace constraints (Sec. 3.4): L per vertex (1 line, 2 plane, 3 none) and
    # the line direction or plane normal; None = no constrained vertex
    sub_dim: Optional[np.ndarray] = None  # (N,) int32
    sub_dir: Optional[np.ndarray] = None  # (N, 3) float64

    @property
    def n_verts(self) -> int:
        return int(self.rest.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


@dataclasses.dataclass
class SimConfig:
    """Simulation parameters shared by both sides (units: SI, +z up)."""

    h: float = 1.0 / 60.0
    iters: int = 20
    steps: int = 100
    gravity: tuple = (0.0, 0.0, -9.8)
    ground_on: bool = False
    ground_height: float = 0.0
    ground_normal: tuple = (0.0, 0.0, 1.0)
    k_c: float = 0.0
    cheby_rho: float = 0.0
    init_mode: int = 3  # 0 previous, 1 inertia, 2 inertia+acceleration, 3 adaptive
    det_eps: float = 1e-12
    k_d: float = 0.0
    mu_c: float = 0.0
    eps_v: float = 1e-3
    line_search: bool = False
    jacobi: bool = False
    self_collision: bool = False
    dcd_radius: float = 0.01
    walls: tuple = ()  # world-box half-spaces (nx, ny, nz, offset): x.n/|n| >= offset
    ccd_interval: int = 0  # vertex-triangle CCD every n_col iterations (with self_collision)
    ccd_edges: bool = False  # that CCD also pairs crossing boundary edges


def world_box(lo, hi) -> list:
    """The six inward-facing walls of the axis-aligned box [lo, hi] as
    (nx, ny, nz, offset) half-spaces, in the order -x, +x, -y, +y, -z, +z
    faces (Sec. 3.4 world-box constraints)."""
    walls = []
    for a in range(3):
        n = [0.0, 0.0, 0.0]
        n[a] = 1.0
        walls.append(tuple(n) + (float(lo[a]),))
        n = [0.0, 0.0, 0.0]
        n[a] = -1.0
        walls.append(tuple(n) + (-float(hi[a]),))
    return walls


def kuhn_grid(nx: int, ny: int, nz: int, edge: float,
              origin=(0.0, 0.0, 0.0)) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Vertices and tets of an nx*ny*nz grid of cubes, 6 tets per cube.

    Vertex (i, j, k) has id i + (nx+1)*(j + (ny+1)*k).  Every cube is split
    along its main diagonal into the 6 tets {c, c+e_a, c+e_a+e_b, c+(1,1,1)}
    over the 6 axis permutations (a, b, c); neighbouring cubes then share
    faces conformingly.
    """
    nxv, nyv, nzv = nx + 1, ny + 1, nz + 1
    k, j, i = np.meshgrid(np.arange(nzv, dtype=np.int32), np.arange(nyv, dtype=np.int32),
                          np.arange(nxv, dtype=np.int32), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    del i, j, k
    rest = np.asarray(origin, dtype=np.float64) + edge * ijk.astype(np.float64)

    # id of each cube's (0,0,0) corner, cubes in x-fastest order (vertex ids
    # fit in int32, so the tables are built in int32 directly)
    if nxv * nyv * nzv >= 2 ** 31:
        raise ValueError("grid too large for int32 vertex ids")
    it = np.int32
    base = (np.arange(nx, dtype=it)[None, None, :] +
            it(nxv) * (np.arange(ny, dtype=it)[None, :, None] +
                       it(nyv) * np.arange(nz, dtype=it)[:, None, None])).ravel()

    def off(e):
        return int(e[0] + nxv * (e[1] + nyv * e[2]))

    unit = np.eye(3, dtype=np.int64)
    table = []
    for perm in itertools.permutations(range(3)):
        e0 = unit[perm[0]]
        e01 = unit[perm[0]] + unit[perm[1]]
        table.append([0, off(e0), off(e01), off((1, 1, 1))])
    table = np.asarray(table, dtype=it)  # (6, 4)
    # cube-major order: the 6 tets of one cube are adjacent
    tets = (base[:, None, None] + table[None, :, :]).reshape(-1, 4)
    return rest, tets, ijk


def kuhn_coloring(ijk: np.ndarray) -> np.ndarray:
    """(i+j+k) mod 4: along each Kuhn tet's lattice path the sum grows by 1,
    so the 4 vertices of every tet get 4 distinct colours."""
    return (ijk.sum(axis=1) % 4).astype(np.int32)


def face_mask(ijk: np.ndarray, dims: tuple, face: str) -> np.ndarray:
    axis = "xyz".index(face[0])
    target = 0 if face[1] == "-" else dims[axis]
    return (ijk[:, axis] == target).astype(np.uint8)


def jitter(rest: np.ndarray, amount: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rest + rng.uniform(-amount, amount, size=rest.shape)


def beam(nx, ny, nz, edge=0.1, E=1e5, nu=0.4, rho=1000.0, pin_face="x-",
         origin=(0.0, 0.0, 0.0), jitter_frac=0.0, seed=0) -> MeshInput:
    rest, tets, ijk = kuhn_grid(nx, ny, nz, edge, origin)
    if jitter_frac > 0:
        rest = jitter(rest, jitter_frac * edge, seed)
    T = tets.shape[0]
    pinned = face_mask(ijk, (nx, ny, nz), pin_face) if pin_face else np.zeros(rest.shape[0], np.uint8)
    return MeshInput(rest=rest, tets=tets,
                     young=np.full(T, E, np.float32), poisson=np.full(T, nu, np.float32),
                     density=np.full(T, rho, np.float32), pinned=pinned, grid_ijk=ijk)


# --------------------------------------------------------------------------
# The workloads.  Sizes follow the scenes of Sec. 5 / Table 1 in shape
# (beam sagging, large drops, many independent bodies, a paper-scale mesh).
# --------------------------------------------------------------------------

def cantilever_beam() -> tuple[MeshInput, SimConfig]:
    """10x3x3 cubes of 0.1 m (176 verts, 540 tets), x=0 face pinned, no ground."""
    m = beam(10, 3, 3, edge=0.1, E=1e5, nu=0.4, rho=1000.0, pin_face="x-")
    return m, SimConfig(h=1 / 60, iters=20, steps=100)


def large_cube(n: int = 100, edge: float = 0.01, seed: int = 1,
               drop_height: float = 0.5) -> tuple[MeshInput, SimConfig]:
    """n^3 cubes, vertices jittered +-10% of the edge, lowest point at
    drop_height above the ground plane z=0 (penalty stiffness 1e7)."""
    rest, tets, ijk = kuhn_grid(n, n, n, edge)
    rest = jitter(rest, 0.1 * edge, seed)
    rest[:, 2] += drop_height - rest[:, 2].min()
    T = tets.shape[0]
    m = MeshInput(rest=rest, tets=tets, young=np.full(T, 1e6, np.float32),
                  poisson=np.full(T, 0.45, np.float32), density=np.full(T, 1000.0, np.float32),
                  pinned=np.zeros(rest.shape[0], np.uint8), grid_ijk=ijk)
    cfg = SimConfig(h=1 / 60, iters=100, steps=20, ground_on=True, k_c=1e7)
    return m, cfg


def paper_scale_cube(n: int = 320, seed: int = 4) -> tuple[MeshInput, SimConfig, np.ndarray]:
    """n^3 cubes (n=320: 33,076,161 verts, 196,608,000 tets) with N(0, 0.5 m/s)
    initial velocities; returns (mesh, config, v0)."""
    m, cfg = large_cube(n, 0.01, seed)
    rng = np.random.default_rng(seed + 1000)
    v0 = rng.normal(0.0, 0.5, size=m.rest.shape)
    cfg.iters, cfg.steps = 20, 5
    return m, cfg, v0


def beam_batch(n_meshes: int = 4096, seed: int = 2, spacing: float = 1.0
               ) -> tuple[list[MeshInput], SimConfig]:
    """Independent beams with cube counts a~U{4..40}, b,c~U{2..8}, edge 0.1 m,
    E log-uniform [1e4, 1e6], nu~U[0.3, 0.48], one random face pinned."""
    rng = np.random.default_rng(seed)
    meshes = []
    for b in range(n_meshes):
        a = int(rng.integers(4, 41))
        bb = int(rng.integers(2, 9))
        c = int(rng.integers(2, 9))
        E = float(np.exp(rng.uniform(np.log(1e4), np.log(1e6))))
        nu = float(rng.uniform(0.3, 0.48))
        face = FACES[int(rng.integers(0, 6))]
        origin = (0.0, spacing * (b % 64), spacing * (b // 64))
        meshes.append(beam(a, bb, c, edge=0.1, E=E, nu=nu, rho=1000.0, pin_face=face, origin=origin))
    return meshes, SimConfig(h=1 / 60, iters=30, steps=50)


def differentiable_beam(seed: int = 3) -> tuple[MeshInput, SimConfig, np.ndarray, np.ndarray]:
    """40x8x8 beam (3,321 verts, 15,360 tets); returns (mesh, cfg, tip_ids, target).
    The target is the rest position of the x=max face plus one seeded offset
    u ~ U[-0.1, 0.1]^3 m."""
    m = beam(40, 8, 8, edge=0.1, E=1e5, nu=0.4, rho=1000.0, pin_face="x-")
    tip = np.nonzero(face_mask(m.grid_ijk, (40, 8, 8), "x+"))[0].astype(np.int64)
    rng = np.random.default_rng(seed)
    target = m.rest[tip] + rng.uniform(-0.1, 0.1, size=3)
    return m, SimConfig(h=1 / 60, iters=50, steps=30), tip, target


def colliding_slabs(n: int = 12, layers: int = 2, edge: float = 0.05, sink: float = 0.1, angle: float = 0.15,
                    seed: int = 7) -> tuple[MeshInput, SimConfig, np.ndarray]:
    """Self-collision workload: a jittered slab of n x n x layers cubes pinned
    at its bottom face, and a free (n-2) x (n-2) x layers slab turned by
    `angle` radians about z and lowered until it overlaps the first by `sink`
    edges (boundary vertices of each end up inside the other).  One body in
    the caller's numbering (the lower slab first); returns (mesh, config,
    index of the first upper-slab vertex)."""
    lower = beam(n, n, layers, edge, E=1e5, nu=0.4, pin_face="z-", jitter_frac=0.05, seed=seed)
    upper = beam(n - 2, n - 2, layers, edge, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.05, seed=seed + 1)
    c, s_ = np.cos(angle), np.sin(angle)
    R = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    centre = upper.rest.mean(axis=0)
    target = np.array([0.5 * n * edge, 0.5 * n * edge, (1.5 * layers - sink) * edge])
    upper.rest = (upper.rest - centre) @ R.T + target
    cat, voff, _ = concat([lower, upper])
    cat.grid_ijk = np.concatenate([lower.grid_ijk, upper.grid_ijk])  # per slab: Kuhn colouring stays valid
    cfg = SimConfig(h=1 / 60, iters=20, steps=10, k_c=1e5, self_collision=True, dcd_radius=0.5 * edge)
    return cat, cfg, int(voff[1])


def concat(meshes: list[MeshInput]) -> tuple[MeshInput, np.ndarray, np.ndarray]:
    """Union of independent meshes plus per-mesh vertex and tet offsets."""
    voff = np.zeros(len(meshes) + 1, np.int64)
    toff = np.zeros(len(meshes) + 1, np.int64)
    for i, m in enumerate(meshes):
        voff[i + 1] = voff[i] + m.n_verts
        toff[i + 1] = toff[i] + m.n_tets
    tets = np.concatenate([m.tets + voff[i] for i, m in enumerate(meshes)]).astype(np.int32)
    cat = MeshInput(rest=np.concatenate([m.rest for m in meshes]), tets=tets,
                    young=np.concatenate([m.young for m in meshes]),
                    poisson=np.concatenate([m.poisson for m in meshes]),
                    density=np.concatenate([m.density for m in meshes]),
                    pinned=np.concatenate([m.pinned for m in meshes]))
    return cat, voff.astype(np.int32), toff.astype(np.int32)


def perturbed_state(rest: np.ndarray, pos_scale: float, vel_scale: float, seed: int
                    ) -> tuple[np.ndarray, np.ndarray]:
    """A deformed configuration and velocities for single-pass checks."""
    rng = np.random.default_rng(seed)
    x = rest + rng.uniform(-pos_scale, pos_scale, size=rest.shape)
    v = rng.normal(0.0, vel_scale, size=rest.shape)
    return x, v


def random_rotation(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
