"""The seeded synthetic workloads match the recipes they stand for (no GPU):
the unit cube, the clamped heterogeneous beam, the 41^3 random lattice the
benchmark times and the 64-lattice batch, with their sizes, materials,
boundary conditions and loads, generated deterministically."""
import numpy as np
import pytest

import synth


def _volumes(s):
    X, T = np.asarray(s.X), np.asarray(s.tets)
    D = np.stack([X[T[:, k]] - X[T[:, 0]] for k in (1, 2, 3)], axis=-1)
    return np.linalg.det(D) / 6.0


def test_cube_recipe():
    """6^3 voxels of the unit cube, six tets each, z = 0 face pinned."""
    s = synth.cube_scene()
    assert (s.n_tets, s.n_verts) == (6 * 6 ** 3, 7 ** 3)
    assert int(s.dirichlet.sum()) == 7 * 7
    assert np.all(s.X[s.dirichlet.astype(bool), 2] == 0.0)
    assert np.allclose(s.X.max(0) - s.X.min(0), 1.0)
    assert np.all(s.E == 1e5) and np.all(s.nu == 0.45) and np.all(s.rho == 1000.0)
    assert s.dt == pytest.approx(1 / 60) and not s.contact
    vol = _volumes(s)
    assert np.all(vol > 0) and vol.sum() == pytest.approx(1.0, rel=1e-12)


def test_beam_recipe():
    """40 x 10 x 10 voxels (1.0 x 0.25 x 0.25 m), x = 0 end clamped, E per
    Voronoi cell from {1e5, 1e9}, nu = 0.4."""
    s = synth.beam_scene()
    assert (s.n_tets, s.n_verts) == (6 * 40 * 10 * 10, 41 * 11 * 11)
    assert int(s.dirichlet.sum()) == 11 * 11
    assert np.all(s.X[s.dirichlet.astype(bool), 0] == s.X[:, 0].min())
    assert np.allclose(s.X.max(0) - s.X.min(0), [1.0, 0.25, 0.25])
    assert set(np.unique(s.E)) == {1e5, 1e9} and np.all(s.nu == 0.4)
    assert np.all(_volumes(s) > 0)


def test_lattice_recipe_of_the_benchmark():
    """41^3 grid, voxels kept with p = 0.55, largest connected component:
    224,226 tets and 72,931 vertices; E log-uniform in [1e5, 1e8] per Voronoi
    cell (32 cells); ground-plane barrier dhat = 1e-3, kappa = 1e5; lifted
    0.05 m and dropped at 1 m/s; no pins."""
    s = synth.lattice_scene(n=41, seed=3, v_down=1.0)
    assert (s.n_tets, s.n_verts) == (224226, 72931)
    kept = s.n_tets / 6 / 41 ** 3
    assert 0.4 < kept <= 0.55 + 0.01            # the largest component of a p = 0.55 draw
    E = np.asarray(s.E)
    assert len(np.unique(E)) == 32 and 1e5 <= E.min() and E.max() <= 1e8
    assert s.contact and s.dhat == 1e-3 and s.kappa == 1e5
    assert s.X[:, 2].min() == pytest.approx(0.05)
    assert np.all(s.v0 == np.array([0.0, 0.0, -1.0])) and not s.dirichlet.any()
    assert np.all(_volumes(s) > 0)
    again = synth.lattice_scene(n=41, seed=3, v_down=1.0)
    assert np.array_equal(again.tets, s.tets) and np.array_equal(again.E, s.E)


def test_batch_of_64_lattices():
    """64 lattices with tet counts log-uniform in [2K, 60K] (before taking the
    largest component), about 1.09M tets in total, binary materials."""
    scenes = synth.batched_lattice_scenes()
    n = np.array([s.n_tets for s in scenes])
    assert len(scenes) == 64
    assert n.sum() == pytest.approx(1.09e6, rel=0.01)
    assert n.min() >= 1000 and n.max() <= 60000
    for s in scenes[::8]:
        assert set(np.unique(s.E)) <= {1e5, 1e9} and s.contact
        assert np.all(_volumes(s) > 0)


def test_lattice_stack_recipe():
    """Two 24^3 lattices (seeds 3 and 4), the lower 0.5 mm above the ground
    at rest, the upper 5 mm above it, shifted (0.3, 0.37) voxels and falling
    at 1 m/s: 89,748 tets, 30,389 vertices; body labels split the vertices;
    no tet mixes bodies."""
    s, body = synth.lattice_stack_scene(24)
    assert (s.n_tets, s.n_verts) == (89748, 30389)
    assert body.shape == (s.n_verts,) and set(np.unique(body)) == {0, 1}
    assert np.all(body[s.tets].min(axis=1) == body[s.tets].max(axis=1))
    lo, hi = s.X[body == 0], s.X[body == 1]
    assert lo[:, 2].min() == pytest.approx(0.0005)
    assert hi[:, 2].min() - lo[:, 2].max() == pytest.approx(0.005)
    assert np.all(s.v0[body == 1] == np.array([0.0, 0.0, -1.0])) and not s.v0[body == 0].any()
    assert s.contact and s.dhat == 1e-3 and s.kappa == 1e5 and not s.dirichlet.any()
    assert np.all(_volumes(s) > 0)
