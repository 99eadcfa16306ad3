"""Seeded voxel tetrahedral meshes.

Every mesh is a voxel set on a regular lattice, each voxel split into six
tetrahedra by the Kuhn (Freudenthal) rule along its (0,0,0)-(1,1,1) diagonal.
The split is conforming across neighbouring voxels because every voxel uses
the same diagonal, and the vertices are the lattice points used by kept
voxels, numbered in lattice order (x fastest, then y, then z).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
from scipy import ndimage

# The six Kuhn tetrahedra of a unit voxel: one per permutation of the axes,
# walking (0,0,0) -> +e_a -> +e_b -> +e_c = (1,1,1).  Odd permutations are
# listed with their middle two vertices swapped so that every tetrahedron is
# positively oriented.
_KUHN = []
for _perm in itertools.permutations(range(3)):
    _c = [(0, 0, 0)]
    _p = [0, 0, 0]
    for _ax in _perm:
        _p = list(_p)
        _p[_ax] += 1
        _c.append(tuple(_p))
    _inv = sum(1 for i in range(3) for j in range(i + 1, 3) if _perm[i] > _perm[j])
    if _inv % 2 == 1:
        _c[1], _c[2] = _c[2], _c[1]
    _KUHN.append(_c)
_KUHN = np.array(_KUHN, dtype=np.int64)  # [6 tets][4 corners][3 offsets]


@dataclass
class Mesh:
    """A tetrahedral mesh: rest positions ``X`` [n,3] f64 and ``tets`` [t,4] i32."""

    X: np.ndarray
    tets: np.ndarray
    lattice_index: np.ndarray  # [n,3] integer lattice coordinates of each vertex
    voxel_of_tet: np.ndarray   # [t] index of the kept voxel each tet came from

    @property
    def n_verts(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def kuhn_voxel_mesh(keep: np.ndarray, voxel: float | tuple = 1.0,
                    origin=(0.0, 0.0, 0.0)) -> Mesh:
    """Mesh the voxels where ``keep[i, j, k]`` is true.

    ``voxel`` is the voxel edge length (a scalar or one length per axis) and
    ``origin`` the position of lattice point (0, 0, 0).
    """
    keep = np.asarray(keep, dtype=bool)
    nx, ny, nz = keep.shape
    h = np.broadcast_to(np.asarray(voxel, dtype=np.float64), (3,))
    vi, vj, vk = np.nonzero(keep)
    # voxel order: x fastest, then y, then z
    order = np.lexsort((vi, vj, vk))
    vi, vj, vk = vi[order], vj[order], vk[order]
    nv = len(vi)
    sx, sy = nx + 1, ny + 1

    def lin(i, j, k):
        return i + sx * (j + sy * k)

    corners = np.empty((nv, 6, 4), dtype=np.int64)
    for t in range(6):
        for c in range(4):
            o = _KUHN[t, c]
            corners[:, t, c] = lin(vi + o[0], vj + o[1], vk + o[2])
    corners = corners.reshape(-1, 4)
    used, inv = np.unique(corners, return_inverse=True)
    tets = inv.reshape(-1, 4).astype(np.int32)
    li = used % sx
    lj = (used // sx) % sy
    lk = used // (sx * sy)
    lat = np.stack([li, lj, lk], axis=1)
    X = np.asarray(origin, dtype=np.float64)[None, :] + lat.astype(np.float64) * h[None, :]
    voxel_of_tet = np.repeat(np.arange(nv), 6)
    return Mesh(X=X, tets=tets, lattice_index=lat, voxel_of_tet=voxel_of_tet)


def lattice_mask(n: int, p: float, seed: int) -> np.ndarray:
    """Random voxel lattice: each voxel of an ``n``^3 grid kept with probability
    ``p`` (seeded), then only the largest 6-connected component retained."""
    rng = np.random.default_rng(seed)
    keep = rng.random((n, n, n)) < p
    lab, nlab = ndimage.label(keep)  # default structure: face (6-) connectivity
    if nlab == 0:
        raise ValueError("empty lattice")
    sizes = np.bincount(lab.ravel())
    sizes[0] = 0
    return lab == int(np.argmax(sizes))


def voronoi_cells(points: np.ndarray, n_cells: int, seed: int,
                  lo=None, hi=None) -> tuple[np.ndarray, np.ndarray]:
    """Assign each point to the nearest of ``n_cells`` seeds drawn uniformly in
    the box [lo, hi] (default: the points' bounding box).  Returns (cell id per
    point, seed positions)."""
    rng = np.random.default_rng(seed)
    lo = points.min(axis=0) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = points.max(axis=0) if hi is None else np.asarray(hi, dtype=np.float64)
    seeds = lo + rng.random((n_cells, 3)) * (hi - lo)
    cell = np.empty(len(points), dtype=np.int64)
    chunk = 65536
    for s in range(0, len(points), chunk):
        d2 = ((points[s:s + chunk, None, :] - seeds[None, :, :]) ** 2).sum(-1)
        cell[s:s + chunk] = np.argmin(d2, axis=1)
    return cell, seeds


def random_tet_mesh(nx: int, ny: int, nz: int, seed: int, jitter: float = 0.15,
                    voxel: float = 0.1) -> Mesh:
    """A small full voxel block whose lattice points are each jittered by up to
    ``jitter`` voxel edges per axis (seeded).  With ``jitter`` <= 0.15 no
    vertex moves past the smallest Kuhn-tet height (0.707 edges) together with
    its neighbour, so every tet keeps its orientation."""
    m = kuhn_voxel_mesh(np.ones((nx, ny, nz), dtype=bool), voxel=voxel)
    rng = np.random.default_rng(seed)
    X = m.X + (rng.random(m.X.shape) - 0.5) * 2.0 * jitter * voxel
    return Mesh(X=X, tets=m.tets, lattice_index=m.lattice_index,
                voxel_of_tet=m.voxel_of_tet)
