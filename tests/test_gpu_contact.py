"""Mesh-mesh contact on the GPU (Eq. IP term B between surface primitives of
different bodies, the CCD filter of Sec. 3.9) against the oracle
(oracle/contact.py, oracle/ip.py with ``body``).

Pins, in the order the path runs: per-pair distance derivatives and the
projected barrier Hessian for every closest-feature type; the broad and
narrow phase against brute force over all pairs (the same set of vertex
tuples); the gradient and H at an iterate with active pairs (fp64 to
rounding, fp32 to float32 storage); the line-search energy and the CCD
bound; whole timesteps of one block driven into another (Jacobi and
two-level PCG) against the oracle's minimiser; and the coarse operator
U^T H U with cross-body blocks against the dense product.
"""
import numpy as np
import pytest

import synth
from oracle import contact, ip, newton

from gpu_helpers import dev, host, rel_disp_error, solver_for, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def _pairs_of_each_type(count=400, seed=3):
    """Random vertex quadruples (both kinds) plus constructed ones that hit
    the interior features: a point above a triangle, crossing edges."""
    r = np.random.default_rng(seed)
    X = r.normal(size=(count, 4, 3))
    kind = r.integers(0, 2, size=count)
    extra_X, extra_k = [], []
    for _ in range(40):
        a, b, c = r.normal(size=(3, 3))
        w = r.dirichlet(np.ones(3))
        n = np.cross(b - a, c - a)
        p = w[0] * a + w[1] * b + w[2] * c + r.normal() * n / np.linalg.norm(n)
        extra_X.append([p, a, b, c])
        extra_k.append(0)
        p0, p1 = r.normal(size=(2, 3))
        m = 0.5 * (p0 + p1) + 0.3 * r.normal(size=3)
        u = r.normal(size=3)
        extra_X.append([p0, p1, m - u, m + u])
        extra_k.append(1)
    return np.concatenate([kind, extra_k]), np.concatenate([X, np.array(extra_X)])


def test_pair_derivatives_match_oracle_for_every_feature():
    from paper_2508_13386_gb300 import contact_pair_derivatives
    kind, X = _pairs_of_each_type()
    dhat, kappa = 10.0, 3.0        # every random pair lies within dhat
    d, g, Hd, Hb = contact_pair_derivatives(kind, X, kappa, dhat)
    seen = set()
    for k in range(len(kind)):
        kk = "pt" if kind[k] == 0 else "ee"
        t = contact._pt_type(*X[k]) if kk == "pt" else contact._ee_type(*X[k])
        seen.add((kk, t[0]))
        d_o, g_o, H_o = contact.pair_distance_derivatives(kk, X[k])
        assert d[k] == pytest.approx(d_o, rel=1e-12)
        assert np.max(np.abs(g[k] - g_o)) <= 1e-10 * np.max(np.abs(g_o))
        assert np.max(np.abs(Hd[k] - H_o)) <= 1e-9 * np.max(np.abs(H_o))
        Hb_o = contact.pair_barrier_hessian(kk, X[k], kappa, dhat)
        assert np.max(np.abs(Hb[k] - Hb_o)) <= 1e-9 * np.max(np.abs(Hb_o))
    assert seen == {("pt", "pt"), ("pt", "pe"), ("pt", "pp"), ("ee", "ee"), ("ee", "pe"), ("ee", "pp")}


def _near_contact(gap_after=4e-4, noise=5e-5, seed=0):
    """The two-block scene with the upper block lowered to gap_after above
    the lower one, positions jittered: pairs within dhat = 1e-3."""
    s, body = synth.two_block_scene(gap=0.004, speed=0.6)
    n0 = int((body == 0).sum())
    x = s.x0.copy()
    x[n0:, 2] -= 0.004 - gap_after
    x += noise * np.random.default_rng(seed).normal(size=x.shape)
    return s, body, x


def _solver(s, body, **opts):
    sol = solver_for(s, **opts)
    sol.set_bodies(body, s.dhat, s.kappa)
    return sol


def _key_pt(q):
    return (int(q[0]), tuple(sorted(int(v) for v in q[1:])))


def _key_ee(q):
    a, b = tuple(sorted(map(int, q[:2]))), tuple(sorted(map(int, q[2:])))
    return tuple(sorted((a, b)))


def test_contact_pairs_match_brute_force():
    """The grid finds exactly the pairs of different bodies within dhat
    (index work: identical sets), and the swept candidates of x -> x + d
    contain every pair within dhat at x, at x + d / 2 and at x + d."""
    s, body, x = _near_contact()
    sol = _solver(s, body)
    pt, ee = sol.contact_pairs(dev(x))
    faces = contact.boundary_faces(s.tets)
    edges = contact.face_edges(faces)
    pt_o, ee_o = contact.contact_pairs(x, faces, edges, body, s.dhat)
    assert len(pt_o) >= 4 and len(ee_o) >= 4
    assert len(pt) == len(pt_o) and len(ee) == len(ee_o)
    assert {_key_pt(q) for q in pt} == {_key_pt([v, *faces[k]]) for v, k in pt_o}
    assert {_key_ee(q) for q in ee} == {_key_ee([*edges[i], *edges[j]]) for i, j in ee_o}
    n0 = int((body == 0).sum())
    d = np.zeros_like(x)
    d[n0:, 2] = -0.0008
    d += 1e-4 * np.random.default_rng(1).normal(size=d.shape)
    spt, see = sol.contact_pairs(dev(x), dev(d))
    cand_pt, cand_ee = {_key_pt(q) for q in spt}, {_key_ee(q) for q in see}
    for xx in (x, x + 0.5 * d, x + d):
        a, b = contact.contact_pairs(xx, faces, edges, body, s.dhat)
        assert {_key_pt([v, *faces[k]]) for v, k in a} <= cand_pt
        assert {_key_ee([*edges[i], *edges[j]]) for i, j in b} <= cand_ee


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_assembly_with_bodies_matches_oracle(precision, tol):
    s, body, x = _near_contact()
    p = ip.Problem(s, body=body)
    sol = _solver(s, body, precision=precision)
    g = host(sol.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt))
    g_o = p.gradient(x)
    assert np.max(np.abs(g - g_o)) <= 1e-11 * np.abs(g_o).max()
    rp, col, val = sol.get_hessian()
    import scipy.sparse as sp
    H = sp.bsr_matrix((val, col, rp), shape=(3 * s.n_verts, 3 * s.n_verts)).toarray()
    H_o = p.hessian(x).toarray()
    assert np.max(np.abs(H - H_o)) <= tol * np.abs(H_o).max()
    # cross-body blocks are present: more blocks than the tet adjacency
    assert len(col) > len({(int(a), int(b)) for t in s.tets for a in t for b in t})


def test_energy_and_ccd_with_bodies_match_oracle():
    s, body, x = _near_contact()
    p = ip.Problem(s, body=body)
    sol = _solver(s, body)
    sol.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt)
    n0 = int((body == 0).sum())
    d = np.zeros_like(x)
    d[n0:, 2] = -0.0006                 # drives the gap (~4e-4) through zero
    d[:n0] = 1e-5 * np.random.default_rng(2).normal(size=(n0, 3))
    a = sol.ccd_bound(dev(x), dev(d))
    a_o = newton.ccd_step_bound(p, x, d)
    assert 0.0 < a_o < 1.0
    assert a == pytest.approx(a_o, rel=1e-9)
    for alpha in (0.0, 0.5 * a_o, a_o):
        E, feasible = sol.energy(dev(x), dev(d), alpha)
        assert feasible
        assert E == pytest.approx(p.energy(x + alpha * d), rel=1e-12)


def test_two_block_collision_step_matches_oracle():
    """One block driven into another (0.6 m/s, 4 mm gap; a free step of
    1/60 s would close it 2.5 times): the CCD-filtered Newton step reaches
    the oracle's minimiser, with the blocks apart."""
    s, body = synth.two_block_scene(gap=0.004, speed=0.6)
    p = ip.Problem(s, body=body)
    x_o, _ = newton.timestep(p)
    sol = _solver(s, body, precision="fp64", newton_tol=1e-10, pcg_rtol=1e-12, max_newton=200)
    dx, st = sol.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert st["status"] == 0 and st["contact_pairs"] > 0
    x1 = s.x0 + host(dx)
    assert rel_disp_error(x1, x_o, s.x0) <= 1e-8
    assert p.feasible(x1)


def test_two_block_two_level_coarse_operator_and_step():
    """Two-level PCG with a basis over both blocks: U^T H U with the
    cross-body blocks equals the dense product of the oracle's H, and the
    step matches the oracle's minimiser."""
    from oracle import subspace
    s, body, x = _near_contact()
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=6, k=3, seed=5)
    p = ip.Problem(s, body=body)
    sol = _solver(s, body, precision="fp64", preconditioner="two_level", newton_tol=1e-10, pcg_rtol=1e-12,
                  max_newton=200)
    sol.upload_basis(origins, vrow, handle, phi)
    sol.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt)
    sol.build_coarse()
    A = sol.get_coarse()
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    A_o = subspace.galerkin(p.hessian(x), U)
    assert np.max(np.abs(A - A_o)) <= 1e-11 * np.abs(A_o).max()
    x_o, _ = newton.timestep(p)
    dx, st = sol.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert st["status"] == 0
    assert rel_disp_error(s.x0 + host(dx), x_o, s.x0) <= 1e-8


def test_two_block_fp32_step_is_close():
    s, body = synth.two_block_scene(gap=0.004, speed=0.6)
    p = ip.Problem(s, body=body)
    x_o, _ = newton.timestep(p)
    sol = _solver(s, body, precision="fp32", newton_tol=1e-6, max_newton=200)
    dx, st = sol.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert st["status"] == 0
    assert rel_disp_error(s.x0 + host(dx), x_o, s.x0) <= 1e-3


def test_set_bodies_rejects_bad_input():
    import paper_2508_13386_gb300 as mls
    s, body = synth.two_block_scene()
    sol = solver_for(s)
    with pytest.raises(mls.MLSError):
        sol.set_bodies(-np.ones(s.n_verts, np.int32), s.dhat, s.kappa)
    with pytest.raises(mls.MLSError):
        sol.set_bodies(body, -1.0, s.kappa)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=6, k=3, seed=5)
    sol.upload_basis(origins, vrow, handle, phi)
    with pytest.raises(mls.MLSError):        # after a basis: rejected
        sol.set_bodies(body, s.dhat, s.kappa)


def test_stack_pairs_sampled_against_brute_force():
    """On the stacked-lattice workload (two 12^3 lattices, the upper one
    lowered into the barrier zone of the lower one, positions jittered) the
    pairs the grid finds for a sample of 300 surface vertices and 300
    surface edges are exactly the oracle's brute-force pairs of those
    primitives with every face or edge of the other body (a box prefilter
    drops only primitives farther than dhat)."""
    s, body = synth.lattice_stack_scene(12)
    x = s.x0.copy()
    up = body == 1
    x[up, 2] -= 0.005 - 4e-4
    x += 5e-5 * np.random.default_rng(4).normal(size=x.shape)
    sol = _solver(s, body)
    pt, ee = sol.contact_pairs(dev(x))
    faces = contact.boundary_faces(s.tets)
    edges = contact.face_edges(faces)
    assert len(pt) > 50 and len(ee) > 100
    r = np.random.default_rng(5)
    sv = np.unique(faces)
    in_pt = np.unique(pt[:, 0])
    vs = np.unique(np.concatenate([r.choice(in_pt, min(200, len(in_pt)), replace=False),
                                 r.choice(sv, 100, replace=False)]))
    flo, fhi = x[faces].min(axis=1) - s.dhat, x[faces].max(axis=1) + s.dhat
    brute = set()
    for v in vs:
        cand = np.nonzero(np.all((flo <= x[v]) & (x[v] <= fhi), axis=1) & (body[faces[:, 0]] != body[v]))[0]
        for k in cand:
            if contact.point_triangle_distance(x[v], *x[faces[k]]) < s.dhat:
                brute.add(_key_pt([v, *faces[k]]))
    found = {_key_pt(q) for q in pt if q[0] in set(vs.tolist())}
    assert found == brute and len(brute) > 30
    eidx = {tuple(e): i for i, e in enumerate(edges)}
    in_ee = np.unique([eidx[tuple(sorted(q[:2]))] for q in ee])
    es = np.unique(np.concatenate([r.choice(in_ee, min(200, len(in_ee)), replace=False),
                                 r.choice(len(edges), 100, replace=False)]))
    elo, ehi = x[edges].min(axis=1), x[edges].max(axis=1)
    brute = set()
    for i in es:
        a, b = edges[i]
        cand = np.nonzero(np.all((elo <= ehi[i] + s.dhat) & (elo[i] - s.dhat <= ehi), axis=1)
                          & (body[edges[:, 0]] != body[a]))[0]
        for j in cand:
            if contact.edge_edge_distance(x[a], x[b], *x[edges[j]]) < s.dhat:
                brute.add(_key_ee([a, b, *edges[j]]))
    sample = {tuple(edges[i]) for i in es}
    found = {_key_ee(q) for q in ee if tuple(sorted(q[:2])) in sample or tuple(sorted(q[2:])) in sample}
    assert found == brute and len(brute) > 50
