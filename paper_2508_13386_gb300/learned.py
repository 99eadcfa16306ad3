"""Training and evaluation of the learned warm start (marshalling only).

Every numeric step runs in the library: the timesteps that generate data
(``mls_newton_step`` with the warm-start history enabled), the features and
targets (``mls_warm_start_sample``), standardisation statistics
(``mls_mlp_column_stats``), training (``mls_mlp_train``, Adam on BF16
tensor-core products) and the warm-started steps.  Python only moves
buffers and draws the seeded random numbers (trajectory loads and minibatch
orders) that the library takes as inputs.

Protocol (the learned-warm-start workload): the beam geometry with a new
material seed; training trajectories each start at rest under a random
gravity (direction within 60 degrees of -z, magnitude 9.81 x U[0.5, 1.5])
with a random initial tip velocity; the network (3r -> 256 -> 256 -> r)
maps [q^t, q^{t-1}, q(h^2 g)] to the Galerkin coarse projection of the
step's increment x^{t+1} - x_tilde; a held-out trajectory
with another seed measures what the warm start saves against the plain
start on the same states.
"""
from __future__ import annotations

import time

import numpy as np


def random_loads(scene, rng):
    """Gravity and initial velocity of one trajectory (seeded inputs)."""
    theta = np.deg2rad(60.0) * np.sqrt(rng.random())
    phi = 2 * np.pi * rng.random()
    mag = 9.81 * rng.uniform(0.5, 1.5)
    g = mag * np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), -np.cos(theta)])
    X = scene.X
    L = X[:, 0].max() - X[:, 0].min()
    s = (X[:, 0] - X[:, 0].min()) / L
    tip = rng.normal(scale=0.5, size=3)
    v0 = s[:, None] ** 2 * tip[None, :]
    v0[np.asarray(scene.dirichlet).astype(bool)] = 0.0
    return g, v0


def drop_loads(scene, rng):
    """Gravity and initial velocity of one trajectory of a free body dropped
    onto the ground plane (seeded inputs): gravity within 30 degrees of -z,
    magnitude 9.81 x U[0.5, 1.5]; a rigid initial velocity, downward speed
    U[0.5, 1.5] m/s, lateral N(0, 0.3) m/s, and a spin N(0, 2) rad/s about
    each axis through the centroid."""
    theta = np.deg2rad(30.0) * np.sqrt(rng.random())
    phi = 2 * np.pi * rng.random()
    mag = 9.81 * rng.uniform(0.5, 1.5)
    g = mag * np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), -np.cos(theta)])
    lin = np.array([rng.normal(scale=0.3), rng.normal(scale=0.3), -rng.uniform(0.5, 1.5)])
    omega = rng.normal(scale=2.0, size=3)
    c = scene.X.mean(axis=0)
    v0 = lin[None, :] + np.cross(omega[None, :], scene.X - c[None, :])
    return g, v0


def scene_loads(scene, rng):
    """The load generator of the scene's kind: clamped bodies (Dirichlet
    vertices) take random_loads, free bodies over a ground plane drop_loads."""
    if np.any(np.asarray(scene.dirichlet)) or not scene.contact:
        return random_loads(scene, rng)
    return drop_loads(scene, rng)


def collect(solver, scene, n_traj, n_steps, seed, device):
    """Run trajectories and return (features [N, 3r], targets [N, r]) as
    float32 CUDA tensors plus per-step solver statistics."""
    import torch
    r = 12 * solver.m
    rng = np.random.default_rng(seed)
    feats = torch.empty(n_traj * n_steps, 3 * r, dtype=torch.float32, device=device)
    targs = torch.empty(n_traj * n_steps, r, dtype=torch.float32, device=device)
    stats = []
    k = 0
    for tr in range(n_traj):
        g, v0 = scene_loads(scene, rng)
        solver.set_forces(tuple(g), scene.contact, scene.plane_n, scene.plane_o, scene.dhat, scene.kappa)
        solver.warm_start_reset()
        x = torch.as_tensor(scene.x0, device=device).contiguous()
        v = torch.as_tensor(v0, device=device).contiguous()
        dx = torch.empty_like(x)
        for _ in range(n_steps):
            _, st = solver.newton_step(x, v, scene.dt, dx=dx)
            solver.warm_start_sample(feats[k], targs[k])
            stats.append(st)
            v.copy_(dx / scene.dt)
            x.add_(dx)
            k += 1
    return feats, targs, stats


def train(mlp, X, T, epochs=60, batch=256, lr=1e-3, seed=0):
    """Standardise with the data's column statistics and train; returns the
    per-epoch mean losses."""
    import torch

    import paper_2508_13386_gb300 as mls
    mx, sx = mls.column_stats(X)
    mt, st = mls.column_stats(T)
    mlp.set_normalization(mx, sx, mt, st)
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    losses = []
    for _ in range(epochs):
        order = torch.as_tensor(rng.permutation(n).astype(np.int32), device=X.device)
        losses.append(mlp.train_epoch(X, T, order, min(batch, n), lr))
    return losses


def evaluate(solver_plain, solver_ws, scene, n_steps, seed, device, recorder=None):
    """Held-out trajectory: the plain solver advances it; the warm-started
    solver takes each step from the same state.  Returns per-step statistics
    of both and the largest relative difference between their results.  With
    a recorder (a third solver with target recording enabled and no network)
    it also takes each step from the same state and returns the held-out
    features and targets, on which the network's prediction error is
    measured."""
    import torch
    rng = np.random.default_rng(seed)
    g, v0 = scene_loads(scene, rng)
    solvers = (solver_plain, solver_ws) + ((recorder,) if recorder is not None else ())
    for s in solvers:
        s.set_forces(tuple(g), scene.contact, scene.plane_n, scene.plane_o, scene.dhat, scene.kappa)
    solver_ws.warm_start_reset()
    feats = targs = None
    if recorder is not None:
        recorder.warm_start_reset()
        r = 12 * recorder.m
        feats = torch.empty(n_steps, 3 * r, dtype=torch.float32, device=device)
        targs = torch.empty(n_steps, r, dtype=torch.float32, device=device)
        dxr = torch.empty_like(torch.as_tensor(scene.x0, device=device))
    x = torch.as_tensor(scene.x0, device=device).contiguous()
    v = torch.as_tensor(v0, device=device).contiguous()
    dxp = torch.empty_like(x)
    dxw = torch.empty_like(x)
    plain, warm = [], []
    worst = 0.0
    tp = tw = 0.0
    for k in range(n_steps):
        if recorder is not None:
            recorder.newton_step(x, v, scene.dt, dx=dxr)
            recorder.warm_start_sample(feats[k], targs[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, sp = solver_plain.newton_step(x, v, scene.dt, dx=dxp)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, sw = solver_ws.newton_step(x, v, scene.dt, dx=dxw)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        tp += t1 - t0
        tw += t2 - t1
        plain.append(sp)
        warm.append(sw)
        den = float(torch.linalg.norm(dxp))
        if den > 0:
            worst = max(worst, float(torch.linalg.norm(dxw - dxp)) / den)
        v.copy_(dxp / scene.dt)
        x.add_(dxp)
    return {"plain": plain, "warm": warm, "max_rel_diff": worst, "plain_s": tp, "warm_s": tw,
            "features": feats, "targets": targs}
