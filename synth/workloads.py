"""The seeded synthetic workloads.

Each builder returns a :class:`Scene`: a mesh, per-tet material parameters
(Young's modulus ``E``, Poisson ratio ``nu``, density ``rho``), a per-vertex
Dirichlet mask, the initial state, gravity, an optional ground plane with its
barrier parameters, and the timestep.  The recipes:

* ``cube_scene``      6^3 unit-cube voxels (1296 tets, 343 verts), E=1e5,
                      nu=0.45, rho=1000, z=0 face pinned, gravity, h=1/60.
* ``beam_scene``      40x10x10 voxels of 0.025 m (24,000 tets), E per seeded
                      Voronoi cell (32 cells) drawn from {1e5, 1e9}, nu=0.4,
                      x=0 face clamped, gravity, h=1/60.
* ``lattice_scene``   n^3 voxels in the unit cube kept with p=0.55, largest
                      6-connected component, lifted 0.05 m above the plane
                      z=0; E log-uniform in [1e5, 1e8] per Voronoi cell
                      (32 cells); nu=0.4; ground barrier dhat=1e-3,
                      kappa=1e5; gravity; h=1/60; optional initial downward
                      speed.  n=41 gives 224,226 tets, n=48 360,126.
* ``batched_lattice_scenes``  64 lattices with tet counts log-uniform in
                      [2K, 60K], materials as the beam, ground barrier.
* ``tiny_scene``      jittered small blocks for unit tests.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .meshes import Mesh, kuhn_voxel_mesh, lattice_mask, voronoi_cells, random_tet_mesh

GRAVITY = (0.0, 0.0, -9.81)


@dataclass
class Scene:
    name: str
    mesh: Mesh
    E: np.ndarray          # [t] Young's modulus, Pa
    nu: np.ndarray         # [t] Poisson ratio
    rho: np.ndarray        # [t] density, kg/m^3
    dirichlet: np.ndarray  # [n] uint8, 1 = pinned at its current position
    x0: np.ndarray         # [n,3] initial positions
    v0: np.ndarray         # [n,3] initial velocities
    dt: float
    gravity: tuple = GRAVITY
    contact: bool = False
    plane_n: tuple = (0.0, 0.0, 1.0)
    plane_o: float = 0.0
    dhat: float = 1e-3
    kappa: float = 1e5
    meta: dict = field(default_factory=dict)

    @property
    def X(self):
        return self.mesh.X

    @property
    def tets(self):
        return self.mesh.tets

    @property
    def n_verts(self):
        return self.mesh.n_verts

    @property
    def n_tets(self):
        return self.mesh.n_tets


def _tet_centroids(mesh: Mesh) -> np.ndarray:
    return mesh.X[mesh.tets].mean(axis=1)


def cube_scene() -> Scene:
    """6x6x6 unit-cube voxel grid, six tets per voxel, bottom face pinned."""
    n = 6
    mesh = kuhn_voxel_mesh(np.ones((n, n, n), dtype=bool), voxel=1.0 / n)
    t = mesh.n_tets
    dirichlet = (mesh.lattice_index[:, 2] == 0).astype(np.uint8)
    return Scene(name="cube6", mesh=mesh, E=np.full(t, 1e5), nu=np.full(t, 0.45),
                 rho=np.full(t, 1000.0), dirichlet=dirichlet, x0=mesh.X.copy(),
                 v0=np.zeros_like(mesh.X), dt=1.0 / 60.0)


def beam_scene(material_seed: int = 2, n_cells: int = 32) -> Scene:
    """40x10x10 voxel beam (1.0 x 0.25 x 0.25 m), x=0 end clamped, E drawn per
    seeded Voronoi cell from {1e5, 1e9} Pa with probability 1/2 each."""
    mesh = kuhn_voxel_mesh(np.ones((40, 10, 10), dtype=bool), voxel=0.025)
    cell, _ = voronoi_cells(_tet_centroids(mesh), n_cells, seed=material_seed,
                            lo=(0, 0, 0), hi=(1.0, 0.25, 0.25))
    rng = np.random.default_rng(material_seed + 1000)
    cell_E = np.where(rng.random(n_cells) < 0.5, 1e5, 1e9)
    t = mesh.n_tets
    dirichlet = (mesh.lattice_index[:, 0] == 0).astype(np.uint8)
    return Scene(name=f"beam40x10x10_s{material_seed}", mesh=mesh, E=cell_E[cell],
                 nu=np.full(t, 0.4), rho=np.full(t, 1000.0), dirichlet=dirichlet,
                 x0=mesh.X.copy(), v0=np.zeros_like(mesh.X), dt=1.0 / 60.0,
                 meta={"material_seed": material_seed})


def lattice_scene(n: int = 41, seed: int = 3, p: float = 0.55, n_cells: int = 32,
                  lift: float = 0.05, materials: str = "loguniform",
                  v_down: float = 0.0) -> Scene:
    """Random voxel lattice in the unit cube ``lift`` above the ground plane
    z=0 with the point-plane log barrier enabled, falling with initial speed
    ``v_down`` (m/s)."""
    keep = lattice_mask(n, p, seed)
    mesh = kuhn_voxel_mesh(keep, voxel=1.0 / n, origin=(0.0, 0.0, lift))
    cell, _ = voronoi_cells(_tet_centroids(mesh), n_cells, seed=seed,
                            lo=(0, 0, lift), hi=(1, 1, 1 + lift))
    rng = np.random.default_rng(seed + 1000)
    if materials == "loguniform":
        cell_E = 10.0 ** rng.uniform(5.0, 8.0, size=n_cells)
    elif materials == "binary":
        cell_E = np.where(rng.random(n_cells) < 0.5, 1e5, 1e9)
    else:
        raise ValueError(materials)
    t = mesh.n_tets
    return Scene(name=f"lattice{n}_p{p}_s{seed}", mesh=mesh, E=cell_E[cell],
                 nu=np.full(t, 0.4), rho=np.full(t, 1000.0),
                 dirichlet=np.zeros(mesh.n_verts, dtype=np.uint8), x0=mesh.X.copy(),
                 v0=np.tile([0.0, 0.0, -v_down], (mesh.n_verts, 1)), dt=1.0 / 60.0, contact=True,
                 meta={"grid": n, "p": p, "seed": seed, "v_down": v_down})


def batched_lattice_scenes(count: int = 64, seed: int = 5, t_min: float = 2e3,
                           t_max: float = 6e4, p: float = 0.55) -> list:
    """``count`` independent lattices whose target tet counts are log-uniform in
    [t_min, t_max]; grid size n = round((t / (6 p))^(1/3))."""
    rng = np.random.default_rng(seed)
    targets = np.exp(rng.uniform(np.log(t_min), np.log(t_max), size=count))
    scenes = []
    for i, tgt in enumerate(targets):
        n = max(3, int(round((tgt / (6.0 * p)) ** (1.0 / 3.0))))
        scenes.append(lattice_scene(n=n, seed=seed * 1000 + i, p=p, materials="binary"))
    return scenes


def tiny_scene(nx: int = 3, ny: int = 2, nz: int = 2, seed: int = 0, contact: bool = False,
               pinned: bool = True, E_range=(1e5, 1e7)) -> Scene:
    """A jittered block of ``nx*ny*nz`` voxels (edge 0.1 m) with per-tet E
    log-uniform in ``E_range``; x=0 face pinned unless ``pinned`` is false."""
    mesh = random_tet_mesh(nx, ny, nz, seed=seed)
    rng = np.random.default_rng(seed + 77)
    t = mesh.n_tets
    E = 10.0 ** rng.uniform(np.log10(E_range[0]), np.log10(E_range[1]), size=t)
    nu = rng.uniform(0.25, 0.45, size=t)
    dirichlet = (mesh.lattice_index[:, 0] == 0).astype(np.uint8) if pinned \
        else np.zeros(mesh.n_verts, dtype=np.uint8)
    lift = 0.0005 if contact else 0.05
    X = mesh.X.copy()
    X[:, 2] += lift - X[:, 2].min()
    mesh = Mesh(X=X, tets=mesh.tets, lattice_index=mesh.lattice_index,
                voxel_of_tet=mesh.voxel_of_tet)
    v0 = rng.normal(scale=0.2, size=X.shape)
    v0[dirichlet.astype(bool)] = 0.0
    return Scene(name=f"tiny{nx}x{ny}x{nz}_s{seed}", mesh=mesh, E=E, nu=nu,
                 rho=np.full(t, 1000.0), dirichlet=dirichlet, x0=X.copy(), v0=v0,
                 dt=1.0 / 60.0, contact=contact)


def two_block_scene(gap: float = 0.01, speed: float = 1.0, seed: int = 0, voxels=(2, 2, 1)):
    """Two separate blocks of ``voxels`` voxels (edge 0.1 m), one above the
    other with ``gap`` between them and a small horizontal offset; the upper
    block moves down at ``speed`` m/s, the lower one rests.  No gravity, no
    ground plane, no pins (a mesh-mesh contact input).  Returns (scene,
    body) with ``body`` [n] the block of each vertex."""
    lower = kuhn_voxel_mesh(np.ones(tuple(voxels), dtype=bool), voxel=0.1)
    upper_X = lower.X + np.array([0.013, -0.007, 0.1 * voxels[2] + gap])
    n0 = lower.n_verts
    X = np.vstack([lower.X, upper_X])
    tets = np.vstack([lower.tets, lower.tets + n0]).astype(np.int32)
    mesh = Mesh(X=X, tets=tets, lattice_index=np.vstack([lower.lattice_index, lower.lattice_index]),
                voxel_of_tet=np.concatenate([lower.voxel_of_tet, lower.voxel_of_tet]))
    t = len(tets)
    v0 = np.zeros_like(X)
    v0[n0:, 2] = -speed
    body = np.concatenate([np.zeros(n0, np.int64), np.ones(n0, np.int64)])
    scene = Scene(name=f"two_blocks_g{gap:g}_v{speed:g}", mesh=mesh, E=np.full(t, 1e5),
                  nu=np.full(t, 0.4), rho=np.full(t, 1000.0), dirichlet=np.zeros(len(X), np.uint8),
                  x0=X.copy(), v0=v0, dt=1.0 / 60.0, gravity=(0.0, 0.0, 0.0), contact=False,
                  dhat=1e-3, kappa=1e5, meta={"seed": seed})
    return scene, body


def lattice_stack_scene(n: int = 24, gap: float = 0.005, speed: float = 1.0, seed: int = 3):
    """Two random voxel lattices (grid ``n`` in the unit cube, p = 0.55,
    materials as ``lattice_scene``, seeds ``seed`` and ``seed + 1``): the
    lower one 0.5 mm above the ground plane z = 0 at rest, the upper one
    ``gap`` above it, shifted by (0.3, 0.37) voxels horizontally so that no
    two parallel surface edges of the two lie within 2 mm of each other,
    falling at ``speed`` m/s.  Gravity, ground barrier dhat = 1e-3,
    kappa = 1e5, h = 1/60.  Returns (scene, body) with ``body`` [n] the
    lattice of each vertex (a mesh-mesh contact workload)."""
    lo = lattice_scene(n=n, seed=seed, lift=0.0005)
    hi = lattice_scene(n=n, seed=seed + 1, lift=0.0)
    top = lo.X[:, 2].max()
    Xh = hi.X.copy()
    Xh[:, 2] += top + gap - Xh[:, 2].min()
    Xh[:, 0] += 0.3 / n
    Xh[:, 1] += 0.37 / n
    n0 = lo.n_verts
    X = np.vstack([lo.X, Xh])
    tets = np.vstack([lo.tets, hi.tets + n0]).astype(np.int32)
    mesh = Mesh(X=X, tets=tets, lattice_index=np.vstack([lo.mesh.lattice_index, hi.mesh.lattice_index]),
                voxel_of_tet=np.concatenate([lo.mesh.voxel_of_tet, hi.mesh.voxel_of_tet]))
    v0 = np.zeros_like(X)
    v0[n0:, 2] = -speed
    body = np.concatenate([np.zeros(n0, np.int64), np.ones(len(X) - n0, np.int64)])
    scene = Scene(name=f"lattice_stack{n}_s{seed}", mesh=mesh, E=np.concatenate([lo.E, hi.E]),
                  nu=np.concatenate([lo.nu, hi.nu]), rho=np.concatenate([lo.rho, hi.rho]),
                  dirichlet=np.zeros(len(X), np.uint8), x0=X.copy(), v0=v0, dt=1.0 / 60.0, contact=True,
                  meta={"grid": n, "seed": seed, "gap": gap, "speed": speed})
    return scene, body


def random_sparse_basis(X: np.ndarray, m: int, k: int, seed: int):
    """A synthetic sparse handle basis for kernel tests (not the paper's
    construction): ``m`` handle origins at random vertices, each vertex tied
    to its ``k`` nearest handles with random positive weights scaled to sum
    to one.  Returns (origins [m,3], vrow [n+1], handle [nnz], phi [nnz])."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    origins = X[rng.choice(n, size=m, replace=False)].copy()
    k = min(k, m)
    d2 = ((X[:, None, :] - origins[None, :, :]) ** 2).sum(-1)
    nearest = np.argsort(d2, axis=1, kind="stable")[:, :k]
    w = rng.random((n, k)) + 0.05
    w /= w.sum(axis=1, keepdims=True)
    order = np.argsort(nearest, axis=1, kind="stable")
    handle = np.take_along_axis(nearest, order, axis=1).astype(np.int32)
    phi = np.take_along_axis(w, order, axis=1)
    vrow = (np.arange(n + 1) * k).astype(np.int32)
    return origins, vrow, handle.ravel(), phi.ravel()


def mlp_init(sizes, seed: int):
    """Initial weights of an MLP with layer widths ``sizes`` (e.g. [in, 256,
    256, out]): W_k [out, in] ~ N(0, 2 / in) (He), biases zero.  Returned as a
    flat list [W1, b1, W2, b2, ...] of float64 arrays."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        params.append(rng.normal(scale=np.sqrt(2.0 / fan_in), size=(fan_out, fan_in)))
        params.append(np.zeros(fan_out))
    return params
