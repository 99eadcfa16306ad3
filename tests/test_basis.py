"""Invariants of the SMS basis construction (Sec. 3.5-3.6), checked on the
host without a GPU: non-negativity, partition of unity with the Dirichlet
basis, interpolation at handles, compact support inside each subdomain,
vanishing at Dirichlet vertices, linear precision, and material awareness
of the partition."""
import numpy as np
import pytest

import synth
from paper_2508_13386_gb300 import basis
from oracle import subspace


def _expand(B, n):
    rows = np.repeat(np.arange(n), np.diff(B["vrow"]))
    return rows, B["handle"], B["phi"]


@pytest.fixture(scope="module")
def beam():
    s = synth.beam_scene()
    return s, basis.build_sms_basis(s.X, s.tets, s.E, 32, dirichlet=s.dirichlet, seed=1)


@pytest.fixture(scope="module")
def beam_heat():
    s = synth.beam_scene()
    return s, basis.build_sms_basis(s.X, s.tets, s.E, 32, dirichlet=s.dirichlet, seed=1, distance="heat")


@pytest.fixture(scope="module")
def lattice():
    s = synth.lattice_scene(n=10, seed=7)
    return s, basis.build_sms_basis(s.X, s.tets, s.E, 12, seed=2)


@pytest.mark.parametrize("which", ["beam", "lattice", "beam_heat"])
def test_partition_of_unity_and_nonnegative(which, request):
    s, B = request.getfixturevalue(which)
    n = s.n_verts
    rows, cols, phi = _expand(B, n)
    assert np.all(phi >= 0)
    tot = np.zeros(n)
    np.add.at(tot, rows, phi)
    assert np.allclose(tot + B["phi_dbc"], 1.0, atol=1e-12)
    free = B["u_dbc"] == 0
    assert np.allclose(tot[free], 1.0, atol=1e-12)


def test_vanishes_at_dirichlet_vertices(beam):
    s, B = beam
    rows, cols, phi = _expand(B, s.n_verts)
    assert np.all(phi[s.dirichlet[rows] == 1] == 0)
    assert np.allclose(B["phi_dbc"][s.dirichlet == 1], 1.0)


@pytest.mark.parametrize("which", ["beam", "lattice", "beam_heat"])
def test_interpolates_at_handles_and_compact_support(which, request):
    s, B = request.getfixturevalue(which)
    n = s.n_verts
    rows, cols, phi = _expand(B, n)
    hv = B["handle_vertex"]
    m = len(hv)
    W = np.zeros((n, m))
    W[rows, cols] = phi
    for i in range(m):
        if B["u_dbc"][hv[i]] == 0:
            assert W[hv[i], i] == pytest.approx(1.0, abs=1e-12)
        for j in B["neighbours"][i]:
            assert W[hv[j], i] == 0.0
        # support within the subdomain (own partition + face neighbours)
        sub = np.isin(B["partition"], [i] + B["neighbours"][i])
        sub_verts = np.unique(s.tets[sub])
        assert np.all(np.isin(np.nonzero(W[:, i])[0], sub_verts))


@pytest.mark.parametrize("which", ["beam", "lattice", "beam_heat"])
def test_linear_precision(which, request):
    """POU weights with affine handle DOFs reproduce any affine map (Sec. 3.5)
    wherever the Dirichlet basis does not take part."""
    s, B = request.getfixturevalue(which)
    rng = np.random.default_rng(5)
    A = rng.normal(size=(3, 3))
    t = rng.normal(size=3)
    U = subspace.lbs_basis_matrix(s.X, B["origins"], B["vrow"], B["handle"], B["phi"])
    q = np.stack([np.concatenate([(A @ o + t)[:, None], A], axis=1).ravel() for o in B["origins"]])
    w = subspace.prolong(U, q)
    free = B["u_dbc"] == 0
    assert np.allclose(w[free], (s.X @ A.T + t)[free], atol=1e-11)


@pytest.mark.parametrize("which", ["beam", "beam_heat"])
def test_partition_is_material_aware(which, request):
    """Stiff regions receive larger partitions than soft ones (Sec. 3.6.1)."""
    s, B = request.getfixturevalue(which)
    vol = np.abs(np.linalg.det(np.stack([s.X[s.tets[:, k]] - s.X[s.tets[:, 0]] for k in (1, 2, 3)], -1))) / 6
    part = B["partition"]
    m = part.max() + 1
    pvol = np.bincount(part, weights=vol, minlength=m)
    stiff_frac = np.bincount(part, weights=vol * (s.E > 1e8), minlength=m) / pvol
    stiff = stiff_frac > 0.3
    soft = stiff_frac < 0.05
    assert stiff.any() and soft.any()
    assert pvol[stiff].mean() > 1.5 * pvol[soft].mean()


def test_handle_count_and_determinism():
    s = synth.cube_scene()
    B1 = basis.build_sms_basis(s.X, s.tets, s.E, 8, dirichlet=s.dirichlet, seed=3)
    B2 = basis.build_sms_basis(s.X, s.tets, s.E, 8, dirichlet=s.dirichlet, seed=3)
    assert len(B1["origins"]) == 8
    assert np.array_equal(B1["handle"], B2["handle"]) and np.array_equal(B1["phi"], B2["phi"])


# ---- heat-method distances (Sec. 3.6) --------------------------------------------------
def test_heat_distance_converges_to_euclidean_in_uniform_material():
    """With one material the metric is Euclidean: the heat-method distance
    from the cube's centre vertex approaches |x - x_s| under refinement, is 0
    at the source and non-negative everywhere."""
    from synth.meshes import kuhn_voxel_mesh
    errs = []
    for nv in (6, 10):
        m = kuhn_voxel_mesh(np.ones((nv, nv, nv), dtype=bool), voxel=1.0 / nv)
        src = int(np.argmin(((m.X - 0.5) ** 2).sum(1)))
        D = basis.HeatDistance(m.X, m.tets, np.ones(m.n_tets))([src])[:, 0]
        E = np.linalg.norm(m.X - m.X[src], axis=1)
        assert D[src] == 0.0 and np.all(D >= 0) and np.all(np.isfinite(D))
        far = E > 0.25
        errs.append(np.mean(np.abs(D[far] - E[far]) / E[far]))
    assert errs[1] < errs[0] and errs[1] < 0.05


def test_heat_distance_follows_the_stiffness_metric():
    """Along a bar whose second half is 16x stiffer, the distance grows at
    the slowness 1/sqrt(k): slope 1 in the soft half and 1/4 in the stiff
    half (the jump-penalty layer at the interface lies between the fits)."""
    from synth.meshes import kuhn_voxel_mesh
    m = kuhn_voxel_mesh(np.ones((24, 3, 3), dtype=bool), voxel=1.0 / 12)
    X, T = m.X, m.tets
    E = np.where(X[T].mean(1)[:, 0] < 1.0, 1e5, 1.6e6)
    _, w_geo = basis.stiffness_weights(T, E)
    src = int(np.argmin(((X - np.array([0.0, 0.125, 0.125])) ** 2).sum(1)))
    line = np.nonzero((np.abs(X[:, 1] - X[src, 1]) < 1e-9) & (np.abs(X[:, 2] - X[src, 2]) < 1e-9))[0]
    D = basis.HeatDistance(X, T, w_geo)([src])[line, 0]
    xs = X[line, 0]
    soft, stiff = (xs > 0.2) & (xs < 0.8), (xs > 1.2) & (xs < 1.8)
    assert np.polyfit(xs[soft], D[soft], 1)[0] == pytest.approx(1.0, rel=0.08)
    assert np.polyfit(xs[stiff], D[stiff], 1)[0] == pytest.approx(0.25, rel=0.05)


def test_heat_kmeans_gives_a_valid_partition():
    s = synth.tiny_scene(6, 4, 3, seed=3)
    labels, centers = basis.kmeans_partition(s.X, s.tets, s.E, 6, seed=2, distance="heat")
    assert len(centers) == 6 and labels.min() == 0 and labels.max() == 5
    assert all(labels[c] == i for i, c in enumerate(centers))
    with pytest.raises(ValueError):
        basis.kmeans_partition(s.X, s.tets, s.E, 6, distance="euclid")


def test_refinement_cg_iterations_counts_edge_hops():
    """Sec. 3.7.2's count: hops from the handle vertex to the farthest vertex
    of its partition through the partition's tets, averaged, binned to 20
    or 40.  On the Kuhn split of a grid a hop moves by any vector of 0/1
    components (or its negative) along the split diagonal, so from the
    centre (2,2,2) of a 4^3-voxel block the farthest vertices, e.g.
    (4,0,0), are 2 + 2 = 4 hops away; along an 80-voxel bar from one end
    the far end is 80 hops away."""
    from paper_2508_13386_gb300 import basis
    cube = synth.kuhn_voxel_mesh(np.ones((4, 4, 4), bool))
    centre = int(np.argmin(((cube.X - 0.5 * cube.X.max(axis=0)) ** 2).sum(1)))
    mean, hops, n_cg = basis.refinement_cg_iterations(cube.tets, np.zeros(len(cube.tets), int), [centre])
    assert hops == [4] and mean == 4.0 and n_cg == 20
    bar = synth.kuhn_voxel_mesh(np.ones((80, 1, 1), bool))
    end = int(np.argmin((bar.X ** 2).sum(1)))
    mean, hops, n_cg = basis.refinement_cg_iterations(bar.tets, np.zeros(len(bar.tets), int), [end])
    assert hops == [80] and n_cg == 40
    # two partitions: the mean of their maxima
    half = (bar.X[bar.tets].mean(axis=1)[:, 0] > bar.X[:, 0].max() / 2).astype(int)
    mid = int(np.argmin(((bar.X - [bar.X[:, 0].max() / 2, 0, 0]) ** 2).sum(1)))
    mean, hops, _ = basis.refinement_cg_iterations(bar.tets, half, [end, mid])
    assert hops == [40, 40] and mean == 40.0
