"""Batched timestep (many independent meshes, one graph launch per step):
each mesh against the oracle timestep from the same state, against the
single-mesh GPU path, the exact special cases, per-mesh status handling and
the 64-mesh lattice workload sampled against the oracle.

Tolerances: the FP64 batch converges every mesh's Newton loop to the step
test 1e-10 and must match the oracle to 1e-9 in the per-step relative
displacement; the FP32 batch (FP32 products and vectors, FP64 reductions)
must match to 1e-4, the bound stated for mixed precision.
"""
import numpy as np
import pytest

import synth
from oracle import ip, newton

from gpu_helpers import rel_disp_error, solver_for, torch

pytestmark = pytest.mark.gpu


def contact_scenes():
    # ragged sizes (no vertex count a multiple of 32), mixed pinning and stiffness
    return [synth.tiny_scene(3, 2, 2, seed=1, contact=True, pinned=False),
            synth.tiny_scene(5, 3, 2, seed=2, contact=True, pinned=False, E_range=(1e5, 1e9)),
            synth.tiny_scene(4, 4, 3, seed=3, contact=True, pinned=True),
            synth.tiny_scene(2, 2, 2, seed=4, contact=True, pinned=False)]


def concat(scenes, attr):
    return np.concatenate([np.asarray(getattr(s, attr), dtype=np.float64) for s in scenes])


def make_batch(scenes, precision, **kw):
    import paper_2508_13386_gb300 as mls
    tol = 1e-10 if precision == "fp64" else 1e-6
    b = mls.Batch(precision=precision, newton_tol=kw.pop("newton_tol", tol), **kw)
    b.upload_scenes(scenes)
    return b


def slices(scenes):
    out, k = [], 0
    for s in scenes:
        out.append(slice(k, k + len(s.X)))
        k += len(s.X)
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_batch_matches_oracle_per_mesh(precision, tol):
    scenes = contact_scenes()
    b = make_batch(scenes, precision)
    x = torch.as_tensor(concat(scenes, "x0"), device="cuda:0")
    v = torch.as_tensor(concat(scenes, "v0"), device="cuda:0")
    dx, stats, info = b.step(x, v, scenes[0].dt)
    assert info["status"] == 0 and info["graph_launches"] == 1
    dxh = dx.cpu().numpy()
    for sc, sl, st in zip(scenes, slices(scenes), stats):
        assert st["status"] == 0 and st["newton_iters"] >= 1
        x_o, _ = newton.timestep(ip.Problem(sc))
        assert rel_disp_error(sc.x0 + dxh[sl], x_o, sc.x0) <= tol


def test_batch_matches_single_mesh_path():
    scenes = contact_scenes()
    b = make_batch(scenes, "fp64")
    x = torch.as_tensor(concat(scenes, "x0"), device="cuda:0")
    v = torch.as_tensor(concat(scenes, "v0"), device="cuda:0")
    dx, stats, _ = b.step(x, v, scenes[0].dt)
    for sc, sl in zip(scenes, slices(scenes)):
        single = solver_for(sc, precision="fp64")
        d1, _ = single.newton_step(torch.as_tensor(sc.x0, device="cuda:0"),
                                   torch.as_tensor(sc.v0, device="cuda:0"), sc.dt)
        a, c = dx[sl].cpu().numpy(), d1.cpu().numpy()
        assert np.linalg.norm(a - c) <= 1e-9 * np.linalg.norm(c)


def test_batch_rest_and_translation_exact():
    """No gravity, no contact: a mesh at rest on a power-of-two voxel grid
    (F = I exactly) has a zero gradient: one Newton iteration and dx = 0
    exactly; a mesh in uniform translation moves by h v (the elastic energy is
    translation invariant)."""
    from synth.meshes import kuhn_voxel_mesh
    from synth.workloads import Scene
    mesh = kuhn_voxel_mesh(np.ones((3, 2, 2), dtype=bool), voxel=0.125, origin=(0.0, 0.0, 0.25))
    t = mesh.n_tets
    rest = Scene(name="rest", mesh=mesh, E=np.full(t, 1e6), nu=np.full(t, 0.3), rho=np.full(t, 1000.0),
                 dirichlet=np.zeros(mesh.n_verts, dtype=np.uint8), x0=mesh.X.copy(),
                 v0=np.zeros_like(mesh.X), dt=1.0 / 60.0, gravity=(0.0, 0.0, 0.0))
    moving = synth.tiny_scene(4, 2, 2, seed=8, pinned=False)
    moving.gravity = (0.0, 0.0, 0.0)
    scenes = [rest, moving]
    b = make_batch(scenes, "fp64")
    v0 = [np.zeros_like(rest.X), np.tile([0.3, -0.2, 0.1], (len(moving.X), 1))]
    x = torch.as_tensor(concat(scenes, "x0"), device="cuda:0")
    v = torch.as_tensor(np.concatenate(v0), device="cuda:0")
    h = rest.dt
    dx, stats, _ = b.step(x, v, h)
    sl = slices(scenes)
    assert stats[0]["newton_iters"] == 1 and stats[0]["status"] == 0
    assert np.all(dx[sl[0]].cpu().numpy() == 0.0)
    assert stats[1]["status"] == 0
    assert np.max(np.abs(dx[sl[1]].cpu().numpy() - h * v0[1])) <= 1e-12


def test_batch_inverted_mesh_fails_alone():
    """A mesh whose x^t has inverted tets reports MLS_EINVERTED; the other
    meshes still complete their steps."""
    scenes = [synth.tiny_scene(3, 2, 2, seed=1, pinned=False), synth.tiny_scene(3, 2, 2, seed=2, pinned=False)]
    b = make_batch(scenes, "fp64")
    x0 = [scenes[0].x0.copy(), scenes[1].x0.copy()]
    x0[0][:, 2] = 2 * x0[0][:, 2].mean() - x0[0][:, 2]     # mirrored: every tet inverted
    x = torch.as_tensor(np.concatenate(x0), device="cuda:0")
    v = torch.as_tensor(concat(scenes, "v0"), device="cuda:0")
    dx, stats, info = b.step(x, v, scenes[0].dt, allow=(-4, -9))
    assert info["status"] == -9
    assert stats[0]["status"] == -9 and stats[1]["status"] == 0
    x_o, _ = newton.timestep(ip.Problem(scenes[1]))
    sl = slices(scenes)[1]
    assert rel_disp_error(scenes[1].x0 + dx[sl].cpu().numpy(), x_o, scenes[1].x0) <= 1e-9


def test_batch_invalid_upload_rejected():
    import paper_2508_13386_gb300 as mls
    s = synth.tiny_scene(2, 2, 2, seed=1)
    b = mls.Batch(precision="fp64")
    T = np.asarray(s.tets)
    with pytest.raises(mls.MLSError):   # a tet of mesh 0 referencing mesh 1
        T2 = np.concatenate([T, T + len(s.X)])
        T2[0, 0] = len(s.X)
        b.upload([0, len(s.X), 2 * len(s.X)], [0, len(T), 2 * len(T)], np.concatenate([s.X, s.X]), T2,
                 np.concatenate([s.E, s.E]), np.concatenate([s.nu, s.nu]), np.concatenate([s.rho, s.rho]))
    with pytest.raises(mls.MLSError):   # an empty mesh
        b.upload([0, len(s.X), len(s.X)], [0, len(T), len(T)], s.X, T, s.E, s.nu, s.rho)


def test_batch_lattice_workload_sampled():
    """The 64-mesh workload (lattices of 2K-60K tets, E in {1e5, 1e9}, ground
    barrier), FP32: three steps from just above the plane, then a fourth step
    compared with the oracle from the same state on the three smallest
    meshes; every mesh must converge."""
    scenes = synth.batched_lattice_scenes()
    drop = np.array([0.0, 0.0, 0.0495])
    for s in scenes:
        s.x0 = s.x0 - drop
    b = make_batch(scenes, "fp32")
    x = torch.as_tensor(concat(scenes, "x0"), device="cuda:0")
    v = torch.zeros_like(x)
    h = scenes[0].dt
    for _ in range(3):
        dx, stats, info = b.step(x, v, h)
        assert all(st["status"] == 0 for st in stats)
        v = dx / h
        x = x + dx
    xs, vs = x.cpu().numpy(), v.cpu().numpy()
    dx, stats, info = b.step(x, v, h)
    assert info["graph_launches"] == 1 and info["spmv_lanes"] in (4, 8)
    assert all(st["status"] == 0 for st in stats)
    sl = slices(scenes)
    order = np.argsort([len(s.tets) for s in scenes])[:3]
    dxh = dx.cpu().numpy()
    for i in order:
        sc = scenes[i]
        p = ip.Problem(sc, x_t=xs[sl[i]], v_t=vs[sl[i]])
        x_o, _ = newton.timestep(p)
        assert rel_disp_error(xs[sl[i]] + dxh[sl[i]], x_o, xs[sl[i]]) <= 1e-4


def random_bases(scenes, k=3, seed=0):
    out = []
    for i, sc in enumerate(scenes):
        m = max(4, int(round(len(sc.tets) / 1400)))
        m = min(m, len(sc.X) // 2)
        o, vr, h, ph = synth.random_sparse_basis(sc.X, m=m, k=min(k, m), seed=seed + i)
        out.append({"origins": o, "vrow": vr, "handle": h, "phi": ph})
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_batch_two_level_matches_oracle_per_mesh(precision, tol):
    """Per-mesh two-level preconditioning (Galerkin U_m^T H_m U_m, float64
    Cholesky per mesh, multiplicative cycle) changes the PCG iterations, not
    the converged step."""
    scenes = contact_scenes()
    b = make_batch(scenes, precision, preconditioner="two_level", omega=0.5)
    b.upload_bases(random_bases(scenes))
    x = torch.as_tensor(concat(scenes, "x0"), device="cuda:0")
    v = torch.as_tensor(concat(scenes, "v0"), device="cuda:0")
    dx, stats, info = b.step(x, v, scenes[0].dt)
    assert info["status"] == 0
    dxh = dx.cpu().numpy()
    for sc, sl, st in zip(scenes, slices(scenes), stats):
        assert st["status"] == 0
        x_o, _ = newton.timestep(ip.Problem(sc))
        assert rel_disp_error(sc.x0 + dxh[sl], x_o, sc.x0) <= tol


def test_batch_two_level_matches_single_mesh_two_level():
    """Same bases through the single-mesh two-level path (coarse operator
    built once per step): same step to 1e-9, and the batch needs far fewer
    PCG iterations than block Jacobi on the stiff mesh."""
    scenes = contact_scenes()
    bases = random_bases(scenes)
    b = make_batch(scenes, "fp64", preconditioner="two_level", omega=0.5)
    b.upload_bases(bases)
    x = torch.as_tensor(concat(scenes, "x0"), device="cuda:0")
    v = torch.as_tensor(concat(scenes, "v0"), device="cuda:0")
    dx, stats, _ = b.step(x, v, scenes[0].dt)
    for sc, sl, B in zip(scenes, slices(scenes), bases):
        single = solver_for(sc, precision="fp64", preconditioner="two_level", cycle="multiplicative", omega=0.5,
                            coarse_refresh=1000)
        single.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
        d1, _ = single.newton_step(torch.as_tensor(sc.x0, device="cuda:0"),
                                   torch.as_tensor(sc.v0, device="cuda:0"), sc.dt)
        a, c = dx[sl].cpu().numpy(), d1.cpu().numpy()
        assert np.linalg.norm(a - c) <= 1e-9 * np.linalg.norm(c)
    bj = make_batch(scenes, "fp64")
    _, stats_j, _ = bj.step(x, v, scenes[0].dt)
    assert stats[1]["pcg_iters"] < stats_j[1]["pcg_iters"]


def test_batch_two_level_lattice_workload_sampled():
    """The 64-mesh workload with per-mesh bases, FP32 two-level: three steps
    from just above the plane, the fourth compared with the oracle on the
    three smallest meshes."""
    scenes = synth.batched_lattice_scenes()
    drop = np.array([0.0, 0.0, 0.0495])
    for s in scenes:
        s.x0 = s.x0 - drop
    b = make_batch(scenes, "fp32", preconditioner="two_level", omega=0.5)
    b.upload_bases(random_bases(scenes, k=4))
    x = torch.as_tensor(concat(scenes, "x0"), device="cuda:0")
    v = torch.zeros_like(x)
    h = scenes[0].dt
    for _ in range(3):
        dx, stats, info = b.step(x, v, h)
        assert all(st["status"] == 0 for st in stats)
        v = dx / h
        x = x + dx
    xs, vs = x.cpu().numpy(), v.cpu().numpy()
    dx, stats, info = b.step(x, v, h)
    assert all(st["status"] == 0 for st in stats)
    sl = slices(scenes)
    dxh = dx.cpu().numpy()
    for i in np.argsort([len(s.tets) for s in scenes])[:3]:
        sc = scenes[i]
        x_o, _ = newton.timestep(ip.Problem(sc, x_t=xs[sl[i]], v_t=vs[sl[i]]))
        assert rel_disp_error(xs[sl[i]] + dxh[sl[i]], x_o, xs[sl[i]]) <= 1e-4
